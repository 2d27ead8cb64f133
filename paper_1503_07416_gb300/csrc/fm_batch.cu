// Batched ensembles: many independent 2-D instances of uneven grid sizes and
// per-instance time steps advance together.  Every stage of the step is one
// launch over all instances (one launch per multigrid level for the level
// work): each launch carries a static work list of (instance, first block)
// items, a block finds its instance by binary search, reads that instance's
// level descriptor, and returns at once if the instance has already
// converged.  The whole step is one CUDA graph with a WHILE node whose
// condition is "some instance is still iterating"; time steps are read from a
// device array, so the graph does not depend on them.
//
// Each instance is a full fm_state (its own arena, hierarchy and, for CDFT,
// kernel transform), so fields, energy and mass are read per instance with
// the single-instance entry points.
#include <cuda_runtime.h>
#include <cstring>
#include <new>
#include <vector>

#include "fm_state.h"
#include "fm_device.cuh"

namespace fm {

struct WorkItem {
  int inst;
  int blk0;
  int aux;   // tiles per row (tile kernels)
  int pad;
};

struct WList {
  int off;      // first item in the item array
  int n;        // items
  int nblocks;  // total blocks
};

template <typename T>
struct InstDev {
  Lvl<T> lv[MAXLEV];
  SmallLv<T> S;
  SmallSmem<T> M;
  InjAll<T> inj_rk;
  InjAll<T> inj_cf;
  Fields64 F;
  Resid64Out O;
  Vel3W velw;
  Vel3 gvel;
  Geo g0;
  double h0;
  double ih0;
  double* partials;
  double* tmp;
  double* rho;
  int nblk64;
  int small_from;
  int nlev;
  int pad;
};

__device__ __forceinline__ int find_item(const WorkItem* it, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (it[mid].blk0 <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool inst_active(const Ctl* ctl, int inst) { return ctl[inst].active != 0; }

// Cooperative copy of a POD struct into shared memory.
template <typename S>
__device__ __forceinline__ void smem_copy(S* dst, const S* src) {
  const int* a = reinterpret_cast<const int*>(src);
  int* b = reinterpret_cast<int*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(S) / sizeof(int)); i += blockDim.x) b[i] = a[i];
}

#define FM_BATCH_HEAD()                                          \
  const int k_ = find_item(items, nitems, blockIdx.x);           \
  const int inst = items[k_].inst;                               \
  const int lb = blockIdx.x - items[k_].blk0;                    \
  (void)lb

// Fused sweep over the tiles of level `level` of all instances (the work list
// maps a tile to its instance; tiles of converged instances are skipped).
// PIPE: persistent blocks over tiles t = blockIdx.x, blockIdx.x + gridDim.x,
// ..., two shared-memory buffers, the next tile's copies in flight while the
// current one is computed; otherwise one tile per block.
template <typename T, int KIND, int TX, int TY, bool SF, bool PIPE, int NS = 1>
__global__ void __launch_bounds__(rb_threads(TX, TY), rb_minb<T>(TX, TY)) kb_smooth_rb2d(const WorkItem* items, int nitems, const InstDev<T>* D,
                                                             const Phys<T>* P, const Ctl* ctl, int level,
                                                             int ntiles, int dir) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* buf0 = reinterpret_cast<T*>(smraw);
  constexpr int BUFSTRIDE = rb_arrays<KIND, SF>() * RBGeom<TX, TY, NS>::SN;
  __shared__ Lvl<T> Gs[2];
  __shared__ int s_inst[2], s_x0[2], s_y0[2];
  int t = blockIdx.x;
  if (t >= ntiles) return;
  auto fetch = [&](int tt, int slot) {
    if (threadIdx.x == 0) {
      const int k = find_item(items, nitems, tt);
      const int inst = items[k].inst;
      const int lb = tt - items[k].blk0;
      const int ntx = items[k].aux;
      s_inst[slot] = inst_active(ctl, inst) ? inst : -1;
      s_x0[slot] = (lb % ntx) * TX;
      s_y0[slot] = (lb / ntx) * TY;
    }
    __syncthreads();
    if (s_inst[slot] >= 0) {
      smem_copy(&Gs[slot], &D[s_inst[slot]].lv[level]);
      __syncthreads();
      rb2d_issue<T, KIND, TX, TY, SF, NS>(Gs[slot], buf0 + slot * BUFSTRIDE, s_x0[slot], s_y0[slot], dir);
    }
    cp_async_commit();
  };
  if constexpr (!PIPE) {
    fetch(t, 0);
    cp_async_wait_all();
    __syncthreads();
    if (s_inst[0] >= 0) rb2d_compute<T, KIND, TX, TY, SF, NS>(Gs[0], P[s_inst[0]], 0, s_x0[0], s_y0[0], dir);
  } else {
    fetch(t, 0);
    for (int k = 0;; ++k) {
      const int tn = t + gridDim.x;
      const bool next = tn < ntiles;
      if (next) fetch(tn, (k + 1) & 1);
      else cp_async_commit();
      cp_async_wait_one();
      __syncthreads();
      const int slot = k & 1;
      if (s_inst[slot] >= 0)
        rb2d_compute<T, KIND, TX, TY, SF, NS>(Gs[slot], P[s_inst[slot]], slot * BUFSTRIDE, s_x0[slot], s_y0[slot],
                                          dir);
      __syncthreads();
      if (!next) break;
      t = tn;
    }
  }
}

// Fused sweep in the row-marching form over the strips of level `level` of
// all instances (work item aux = strips per row of blocks).
template <typename T, int KIND, int TX>
__global__ void __launch_bounds__(march_threads(TX), march_minb<T>(TX)) kb_smooth_march(const WorkItem* items, int nitems,
                                                                     const InstDev<T>* D, const Phys<T>* P,
                                                                     const Ctl* ctl, int level, int ly, int dir) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ Lvl<T> Gs;
  FM_BATCH_HEAD();
  if (!inst_active(ctl, inst)) return;
  smem_copy(&Gs, &D[inst].lv[level]);
  __syncthreads();
  const int nstrips = items[k_].aux;
  const int strip = lb % nstrips, seg = lb / nstrips;
  const int y0 = seg * ly;
  march_sweep<T, KIND, TX>(Gs, P[inst], reinterpret_cast<T*>(smraw), strip * TX, y0, min(y0 + ly, Gs.g.ny), dir);
}

// Two sweeps per pass in the row-marching form (see k_smooth_march2) over the
// strips of level `level` of all instances (work item aux = strips per row).
template <typename T, int KIND, int TX>
__global__ void __launch_bounds__(march_threads(TX), march2_minb<T>(TX)) kb_smooth_march2(const WorkItem* items, int nitems,
                                                                      const InstDev<T>* D, const Phys<T>* P,
                                                                      const Ctl* ctl, int level, int ly, int dir) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ Lvl<T> Gs;
  FM_BATCH_HEAD();
  if (!inst_active(ctl, inst)) return;
  smem_copy(&Gs, &D[inst].lv[level]);
  __syncthreads();
  const int nstrips = items[k_].aux;
  const int strip = lb % nstrips, seg = lb / nstrips;
  const int y0 = seg * ly;
  march2_sweep<T, KIND, TX>(Gs, P[inst], reinterpret_cast<T*>(smraw), strip * TX, y0, min(y0 + ly, Gs.g.ny), dir);
}

// Exchange the correction and residual buffers of a level held in shared
// memory (block-uniform `swap`; the correction is in r).
template <typename T>
__device__ __forceinline__ void lvl_swap_er(Lvl<T>& L, int swap) {
  if (!swap) return;
  if (threadIdx.x < MAXU) {
    T* t = L.e[threadIdx.x];
    L.e[threadIdx.x] = L.r[threadIdx.x];
    L.r[threadIdx.x] = t;
  }
  __syncthreads();
}

// e = r at every point of level `level` (after an odd number of fused sweeps).
template <typename T, int NU>
__global__ void __launch_bounds__(TPB) kb_copy_back(const WorkItem* items, int nitems, const InstDev<T>* D,
                                                    const Ctl* ctl, int level) {
  FM_BATCH_HEAD();
  if (!inst_active(ctl, inst)) return;
  const Lvl<T>& L = D[inst].lv[level];
  const int idx = lb * TPB + threadIdx.x;
  if (idx >= L.g.N) return;
#pragma unroll
  for (int q = 0; q < NU; ++q) L.e[q][idx] = L.r[q][idx];
}

// Fine residual and restriction of level `level` in one launch (see
// k_resid_restrict2); work item aux = coarse tiles per row.  fswap: the fine
// correction is in the level's r buffer.
template <typename T, int KIND>
__global__ void __launch_bounds__(TPB) kb_resid_restrict2(const WorkItem* items, int nitems, const InstDev<T>* D,
                                                          const Phys<T>* P, const Ctl* ctl, int level, int fswap) {
  FM_BATCH_HEAD();
  if (!inst_active(ctl, inst)) return;
  __shared__ Lvl<T> F, Cc;
  __shared__ T sr[Layout<KIND, 2>::NU * RR_FN];
  smem_copy(&F, &D[inst].lv[level]);
  smem_copy(&Cc, &D[inst].lv[level + 1]);
  __syncthreads();
  lvl_swap_er(F, fswap);
  const int ntx = items[k_].aux;
  resid_restrict2_tile<T, KIND>(F, Cc, P[inst], (lb % ntx) * RR_TX, (lb / ntx) * RR_TY, sr);
}

template <typename T, int NU>
__global__ void __launch_bounds__(TPB) kb_prolong(const WorkItem* items, int nitems, const InstDev<T>* D,
                                                  const Phys<T>* P, const Ctl* ctl, int level, int fswap) {
  FM_BATCH_HEAD();
  if (!inst_active(ctl, inst)) return;
  __shared__ Lvl<T> F, Cc;
  smem_copy(&F, &D[inst].lv[level]);
  smem_copy(&Cc, &D[inst].lv[level + 1]);
  __syncthreads();
  lvl_swap_er(F, fswap);
  const int idx = lb * TPB + threadIdx.x;
  if (idx < F.g.N) prolong_point<T, NU, 2>(F, Cc, P[inst], idx);
}

// one block per instance
template <typename T, int KIND>
__global__ void __launch_bounds__(SMALL_TPB) kb_small(const InstDev<T>* D, const Phys<T>* P, const Ctl* ctl,
                                                      int nu1, int nu2, int ncoarse) {
  const int inst = blockIdx.x;
  if (!inst_active(ctl, inst)) return;
  vcycle_small_smem_body<T, KIND, 2>(D[inst].S, D[inst].M, P[inst], nu1, nu2, ncoarse);
}

// Same, data in global memory (small levels too large for shared memory).
template <typename T, int KIND>
__global__ void __launch_bounds__(SMALL_TPB) kb_small_global(const InstDev<T>* D, const Phys<T>* P,
                                                             const Ctl* ctl, int nu1, int nu2, int ncoarse) {
  const int inst = blockIdx.x;
  if (!inst_active(ctl, inst)) return;
  vcycle_small_body<T, KIND, 2>(D[inst].S, P[inst], nu1, nu2, ncoarse);
}

template <typename T>
__global__ void __launch_bounds__(TPB) kb_inject(const WorkItem* items, int nitems, const InstDev<T>* D,
                                                 const Ctl* ctl, int coefficients, int check_active) {
  FM_BATCH_HEAD();
  if (check_active && !inst_active(ctl, inst)) return;
  const InjAll<T>& A = coefficients ? D[inst].inj_cf : D[inst].inj_rk;
  inject_all_point<T>(A, lb * TPB + threadIdx.x);
}

template <typename T, int KIND>
__global__ void __launch_bounds__(TPB) kb_prepare(const WorkItem* items, int nitems, const InstDev<T>* D,
                                                  const Phys<double>* P64, const Step64* K64) {
  FM_BATCH_HEAD();
  prepare_point<KIND, 2>(D[inst].F, D[inst].g0, K64[inst], P64[inst], lb * TPB + threadIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(TPB) kb_prepare_mu(const WorkItem* items, int nitems, const InstDev<T>* D,
                                                     const Phys<double>* P64, const Step64* K64) {
  FM_BATCH_HEAD();
  prepare_mu_point<2>(D[inst].F, D[inst].g0, K64[inst], P64[inst], lb * TPB + threadIdx.x);
}

template <typename T, int KIND>
__global__ void __launch_bounds__(TPB) kb_resid64(const WorkItem* items, int nitems, const InstDev<T>* D,
                                                  const Phys<double>* P64, const Step64* K64, const Ctl* ctl,
                                                  int check_active) {
  FM_BATCH_HEAD();
  if (check_active && !inst_active(ctl, inst)) return;
  const InstDev<T>& I = D[inst];
  resid64_tile_body<KIND, T>(I.F, I.O, I.g0, K64[inst], P64[inst], I.partials, lb, I.nblk64);
}

// one block per instance: norm, cycles, status, active flag
template <typename T, int NQ>
__global__ void kb_norm(const InstDev<T>* D, Ctl* ctl, double tol, int max_cycles, int in_body) {
  const int inst = blockIdx.x;
  if (in_body && !inst_active(ctl, inst)) return;
  const InstDev<T>& I = D[inst];
  const double w = I.h0 * I.h0;
  const bool cont = norm_ctl_body<NQ>(I.partials, I.nblk64, w, &ctl[inst], tol, max_cycles, in_body);
  if (threadIdx.x == 0) ctl[inst].active = cont ? 1 : 0;
}

__global__ void kb_set_active(Ctl* ctl, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    ctl[i].active = 1;
    ctl[i].nonpos = 0;
  }
}

__global__ void kb_condition(const Ctl* ctl, int count, cudaGraphConditionalHandle handle) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x)
    if (ctl[i].active) atomicOr(&any, 1);
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(handle, any ? 1u : 0u);
}

template <typename T, int NU>
__global__ void __launch_bounds__(TPB) kb_update64(const WorkItem* items, int nitems, const InstDev<T>* D,
                                                   const Ctl* ctl, double delta) {
  FM_BATCH_HEAD();
  if (!inst_active(ctl, inst)) return;
  const InstDev<T>& I = D[inst];
  update64_point<NU, T>(I.F, I.O, I.g0.N, delta, lb * TPB + threadIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(TPB) kb_closure(const WorkItem* items, int nitems, const InstDev<T>* D,
                                                  const Phys<double>* P64, const Step64* K64, const Ctl* ctl) {
  FM_BATCH_HEAD();
  if (ctl[inst].status != FM_OK) return;
  const InstDev<T>& I = D[inst];
  closure_point<2>(I.F, I.g0, K64[inst], P64[inst], I.tmp, lb * TPB + threadIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(TPB) kb_commit(const WorkItem* items, int nitems, const InstDev<T>* D,
                                                 const Ctl* ctl) {
  FM_BATCH_HEAD();
  if (ctl[inst].status != FM_OK) return;
  const InstDev<T>& I = D[inst];
  commit_point<2>(I.rho, I.velw, I.tmp, I.gvel, I.g0.N, lb * TPB + threadIdx.x);
}

}  // namespace fm

using namespace fm;

struct fm_batch {
  int count;
  int kind;
  fm_params prm;
  fm_functional fn;
  fm_state** inst;
  int maxdepth;              // max over instances of small_from (levels handled level by level)
  size_t small_smem;         // dynamic shared memory of the small-level kernel
  bool small_global;         // small levels too large for shared memory: global-memory kernel
  // device tables
  void* dev;                 // one allocation: descriptors, phys, ctl, work items
  void* D;                   // InstDev<T>[count]
  void* P;                   // Phys<T>[count]
  Phys<double>* P64;
  Step64* K64;               // float64 step constants per instance
  Ctl* ctl;
  WorkItem* items;
  // host staging (pinned)
  void* hP;
  Phys<double>* hP64;
  Step64* hK64;
  Ctl* hctl;
  // work lists
  std::vector<WorkItem> hitems;
  WList w_fine, w_resid64, w_inject;
  WList w_smooth[3 + 6][MAXLEV];  // per tile shape (32x16, 64x8, 32x32), then per marching variant
  WList w_resid[MAXLEV], w_rr[MAXLEV], w_prolong[MAXLEV];
  int rbv[MAXLEV];           // chosen fused-sweep variant per level
  float rbt[MAXLEV][RB_NVAR];  // autotuner timings (ms per sweep)
  // graph
  cudaStream_t stream;
  cudaStream_t user_stream;
  cudaStream_t cap[2];
  cudaGraph_t graph;
  cudaGraphExec_t gexec;
  long long cnt_pre, cnt_body, cnt_post, launches;
};

namespace fm {

#define FMB_CUDA(call)                         \
  do {                                         \
    if ((call) != cudaSuccess) {               \
      cudaGetLastError();                      \
      return FM_ECUDA;                         \
    }                                          \
  } while (0)

#define FMB_LAUNCHED()                         \
  do {                                         \
    ++b->launches;                             \
    if (cudaPeekAtLastError() != cudaSuccess) { \
      cudaGetLastError();                      \
      return FM_ECUDA;                         \
    }                                          \
  } while (0)

static WList add_list(fm_batch* b, const std::vector<std::pair<int, int>>& inst_blocks,
                      const std::vector<int>* aux = nullptr) {
  WList w;
  w.off = (int)b->hitems.size();
  w.n = 0;
  w.nblocks = 0;
  for (size_t i = 0; i < inst_blocks.size(); ++i) {
    if (inst_blocks[i].second <= 0) continue;
    WorkItem it;
    it.inst = inst_blocks[i].first;
    it.blk0 = w.nblocks;
    it.aux = aux ? (*aux)[i] : 0;
    it.pad = 0;
    b->hitems.push_back(it);
    w.nblocks += inst_blocks[i].second;
    ++w.n;
  }
  return w;
}

template <typename T, int KIND>
struct Batch {
  using LY = Layout<KIND, 2>;

  static void build_desc(fm_batch* b, std::vector<InstDev<T>>& H) {
    for (int i = 0; i < b->count; ++i) {
      fm_state* st = b->inst[i];
      InstDev<T>& I = H[i];
      memset(&I, 0, sizeof(I));
      for (int l = 0; l < st->nlev; ++l) I.lv[l] = make_lvl<T>(st, l);
      I.nlev = st->nlev;
      I.small_from = st->small_from;
      // small levels and their shared-memory layout
      I.S.count = st->nlev - st->small_from;
      for (int q = 0; q < I.S.count; ++q) I.S.lv[q] = make_lvl<T>(st, st->small_from + q);
      const size_t smb = small_layout<T, KIND, 2>(I.S, I.M, SMALL_SMEM_MAX);
      if (smb > b->small_smem) b->small_smem = smb;
      if (I.S.lv[0].g.N > SMALL_SMEM_N) b->small_global = true;
      // injections (all coarse levels at once)
      for (int which = 0; which < 2; ++which) {
        InjAll<T>& A = which ? I.inj_cf : I.inj_rk;
        A.nl = st->nlev;
        A.g0 = st->lv[0].g;
        A.off[0] = A.off[1] = 0;
        for (int l = 1; l < st->nlev; ++l) {
          A.g[l] = st->lv[l].g;
          A.off[l + 1] = A.off[l] + st->lv[l].g.N;
        }
        int q = 0;
        if (which) {
          A.src[q] = (const T*)st->lv[0].cr;
          for (int l = 1; l < st->nlev; ++l) A.dst[l][q] = (T*)st->lv[l].cr;
          ++q;
          for (int d = 0; d < 2; ++d, ++q) {
            A.src[q] = (const T*)st->lv[0].cv[d];
            for (int l = 1; l < st->nlev; ++l) A.dst[l][q] = (T*)st->lv[l].cv[d];
          }
        } else {
          A.src[q] = (const T*)st->lv[0].rk;
          for (int l = 1; l < st->nlev; ++l) A.dst[l][q] = (T*)st->lv[l].rk;
          ++q;
          A.src[q] = (const T*)st->lv[0].om[0];
          for (int l = 1; l < st->nlev; ++l) A.dst[l][q] = (T*)st->lv[l].om[0];
          ++q;
        }
        A.nsrc = q;
      }
      I.F = make_fields(st);
      for (int q = 0; q < MAXU; ++q) {
        I.O.f0[q] = q < LY::NU ? st->lv[0].f[q] : nullptr;
        I.O.e0[q] = q < LY::NU ? st->lv[0].e[q] : nullptr;
        I.O.r64[q] = nullptr;
      }
      I.O.cr32 = nullptr;
      for (int d = 0; d < 3; ++d) I.O.cv32[d] = nullptr;
      if (b->prm.precision == FM_MIXED) {
        I.O.cr32 = (float*)st->lv[0].cr;
        for (int d = 0; d < 2; ++d) I.O.cv32[d] = (float*)st->lv[0].cv[d];
      }
      I.velw = Vel3W{{st->vel[0], st->vel[1], nullptr}};
      I.gvel = Vel3{{st->g[1], st->g[2], nullptr}};
      I.g0 = st->lv[0].g;
      I.h0 = st->lv[0].h;
      I.ih0 = 1.0 / st->lv[0].h;
      I.partials = st->partials;
      I.tmp = st->tmp;
      I.rho = st->rho;
      I.nblk64 = st->nblk;
    }
  }

  static void build_lists(fm_batch* b) {
    std::vector<std::pair<int, int>> v;
    b->maxdepth = 0;
    for (int i = 0; i < b->count; ++i)
      if (b->inst[i]->small_from > b->maxdepth) b->maxdepth = b->inst[i]->small_from;
    // finest points, float64 residual blocks, coarse injection points
    v.clear();
    for (int i = 0; i < b->count; ++i) v.push_back({i, nblocks(b->inst[i]->lv[0].g.N)});
    b->w_fine = add_list(b, v);
    v.clear();
    for (int i = 0; i < b->count; ++i) v.push_back({i, b->inst[i]->nblk});
    b->w_resid64 = add_list(b, v);
    v.clear();
    for (int i = 0; i < b->count; ++i) {
      long long n = 0;
      for (int l = 1; l < b->inst[i]->nlev; ++l) n += b->inst[i]->lv[l].g.N;
      v.push_back({i, nblocks(n)});
    }
    b->w_inject = add_list(b, v);
    for (int l = 0; l < b->maxdepth; ++l) {
      std::vector<std::pair<int, int>> ts[9], rs, cr, pr;
      std::vector<int> aux[9], craux;
      for (int i = 0; i < b->count; ++i) {
        fm_state* st = b->inst[i];
        if (st->small_from <= l) continue;
        const Geo g = st->lv[l].g, gc = st->lv[l + 1].g;
        for (int sh = 0; sh < 3; ++sh) {
          const int TX = sh == 1 ? 64 : 32, TY = sh == 0 ? 16 : (sh == 1 ? 8 : 32);
          const int ntx = (g.nx + TX - 1) / TX, nty = (g.ny + TY - 1) / TY;
          ts[sh].push_back({i, ntx * nty});
          aux[sh].push_back(ntx);
        }
        for (int m = 0; m < 6; ++m) {  // marching variants RB_NTILE + m
          const int TX = march_tx(RB_NTILE + m), LYR = march_ly(RB_NTILE + m);
          const int nstrips = (g.nx + TX - 1) / TX, nseg = (g.ny + LYR - 1) / LYR;
          ts[3 + m].push_back({i, nstrips * nseg});
          aux[3 + m].push_back(nstrips);
        }
        rs.push_back({i, nblocks(g.N)});
        const int ctx = (gc.nx + RR_TX - 1) / RR_TX, cty = (gc.ny + RR_TY - 1) / RR_TY;
        cr.push_back({i, ctx * cty});  // coarse tiles of the fused residual + restriction
        craux.push_back(ctx);
        pr.push_back({i, nblocks(g.N)});
      }
      for (int sh = 0; sh < 9; ++sh) b->w_smooth[sh][l] = add_list(b, ts[sh], &aux[sh]);
      b->w_resid[l] = add_list(b, rs);
      b->w_rr[l] = add_list(b, cr, &craux);
      b->w_prolong[l] = add_list(b, pr);
    }
  }

  static const WorkItem* it(fm_batch* b, const WList& w) { return b->items + w.off; }

  template <int TX, int TY, bool SF, bool PIPE, int NS = 1>
  static int launch_v(fm_batch* b, int l, int dir) {
    constexpr size_t smem = rb_smem_bytes<T, KIND, TX, TY, SF, PIPE, NS>();
    if (smem + 4096 > (size_t)b->inst[0]->smem_optin) return FM_EINVAL;  // does not fit: skip
    static int per_sm = 0;
    if (!per_sm) {
      FMB_CUDA(cudaFuncSetAttribute(kb_smooth_rb2d<T, KIND, TX, TY, SF, PIPE, NS>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      FMB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_smooth_rb2d<T, KIND, TX, TY, SF, PIPE, NS>,
                                                             rb_threads(TX, TY), smem));
      if (per_sm < 1) per_sm = 1;
    }
    const WList& w = b->w_smooth[TX == 64 ? 1 : (TY == 32 ? 2 : 0)][l];
    int grid = w.nblocks;
    if (PIPE && grid > per_sm * b->inst[0]->sms) grid = per_sm * b->inst[0]->sms;
    kb_smooth_rb2d<T, KIND, TX, TY, SF, PIPE, NS><<<grid, rb_threads(TX, TY), smem, b->stream>>>(
        it(b, w), w.n, (const InstDev<T>*)b->D, (const Phys<T>*)b->P, b->ctl, l, w.nblocks, dir);
    FMB_LAUNCHED();
    return FM_OK;
  }

  // Marching form, variant v (strip width TX) over all instances.
  template <int TX>
  static int launch_m(fm_batch* b, int l, int dir, int v) {
    constexpr size_t smem = march_smem_bytes<T, KIND, TX>();
    if (smem + 4096 > (size_t)b->inst[0]->smem_optin) return FM_EINVAL;  // does not fit: skip
    static bool attr = false;
    if (!attr) {
      FMB_CUDA(cudaFuncSetAttribute(kb_smooth_march<T, KIND, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
      attr = true;
    }
    const WList& w = b->w_smooth[3 + v - RB_NTILE][l];
    kb_smooth_march<T, KIND, TX><<<w.nblocks, march_threads(TX), smem, b->stream>>>(
        it(b, w), w.n, (const InstDev<T>*)b->D, (const Phys<T>*)b->P, b->ctl, l, march_ly(v), dir);
    FMB_LAUNCHED();
    return FM_OK;
  }

  // Two-sweep marching form, variant v (strip width TX) over all instances.
  template <int TX>
  static int launch_m2(fm_batch* b, int l, int dir, int v) {
    constexpr size_t smem = march2_smem_bytes<T, KIND, TX>();
    if (smem + 4096 > (size_t)b->inst[0]->smem_optin) return FM_EINVAL;  // does not fit: skip
    static bool attr = false;
    if (!attr) {
      FMB_CUDA(cudaFuncSetAttribute(kb_smooth_march2<T, KIND, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
      attr = true;
    }
    const WList& w = b->w_smooth[3 + (v - RB_NTILE) % RB_NMARCH][l];
    kb_smooth_march2<T, KIND, TX><<<w.nblocks, march_threads(TX), smem, b->stream>>>(
        it(b, w), w.n, (const InstDev<T>*)b->D, (const Phys<T>*)b->P, b->ctl, l, march_ly(v), dir);
    FMB_LAUNCHED();
    return FM_OK;
  }

  static int launch_variant(fm_batch* b, int v, int l, int dir = 0) {
    switch (v) {
      case 0: return launch_v<32, 16, false, false>(b, l, dir);
      case 1: return launch_v<32, 16, false, true>(b, l, dir);
      case 2: return launch_v<32, 16, true, false>(b, l, dir);
      case 3: return launch_v<32, 16, true, true>(b, l, dir);
      case 4: return launch_v<64, 8, false, false>(b, l, dir);
      case 5: return launch_v<64, 8, false, true>(b, l, dir);
      case 6: return launch_v<64, 8, true, false>(b, l, dir);
      case 7: return launch_v<64, 8, true, true>(b, l, dir);
      case 8: return launch_v<32, 32, false, false>(b, l, dir);
      case 9: return launch_v<32, 32, false, true>(b, l, dir);
      case 10: return launch_v<32, 32, true, false>(b, l, dir);
      case 11: return launch_v<32, 32, true, true>(b, l, dir);
      case 12: return launch_m<64>(b, l, dir, 12);
      case 13: return launch_m<64>(b, l, dir, 13);
      case 14: return launch_m<64>(b, l, dir, 14);
      case 15: return launch_m<128>(b, l, dir, 15);
      case 16: return launch_m<128>(b, l, dir, 16);
      case 17: return launch_m<128>(b, l, dir, 17);
      case 18: return launch_m2<64>(b, l, dir, 18);
      case 19: return launch_m2<64>(b, l, dir, 19);
      case 20: return launch_m2<64>(b, l, dir, 20);
      case 21: return launch_m2<128>(b, l, dir, 21);
      case 22: return launch_m2<128>(b, l, dir, 22);
      case 23: return launch_m2<128>(b, l, dir, 23);
      case 24: return launch_v<32, 16, false, false, 2>(b, l, dir);
      case 25: return launch_v<64, 8, false, false, 2>(b, l, dir);
      // 27..29 (tile staging by tensor copies in the single-instance
      // solver): the same tiles staged by cp.async here
      case 27: return launch_v<32, 16, false, false, 2>(b, l, dir);
      case 28: return launch_v<32, 16, false, false>(b, l, dir);
      // 30..33 (small tiles in the single-instance solver): the 32 x 16 tiles here
      case 30: return launch_v<32, 16, false, false>(b, l, dir);
      case 31: return launch_v<32, 16, false, false, 2>(b, l, dir);
      case 32: return launch_v<32, 16, false, false>(b, l, dir);
      case 33: return launch_v<32, 16, false, false, 2>(b, l, dir);
      case 34: return launch_v<32, 16, false, false, 2>(b, l, dir);  // (cooperative in the single solver)
      case 35: return launch_v<32, 16, false, false, 2>(b, l, dir);  // (32 x 14 tiles in the single solver)
      default: return launch_v<32, 32, false, false, 2>(b, l, dir);
    }
  }

  // `iters` sweeps of level l.  Each launch reads the correction from one
  // buffer and writes it to the other; *in_r says (and is updated to) whether
  // it is in r.  A two-sweep variant runs the sweeps in pairs and an odd last
  // sweep with the one-sweep variant of the same blocks.
  static int smooth(fm_batch* b, int l, int iters, int* in_r) {
    if (b->w_smooth[0][l].n == 0) return FM_OK;
    const int v = b->rbv[l];
    for (int k = 0; k < iters;) {
      const int two = sweeps_per_launch(v) == 2 && k + 2 <= iters;
      const int rc = launch_variant(b, (sweeps_per_launch(v) == 2 && !two) ? one_sweep_twin(v) : v, l, *in_r);
      if (rc) return rc;
      *in_r ^= 1;
      k += two ? 2 : 1;
    }
    return FM_OK;
  }

  static int copy_back(fm_batch* b, int l) {
    const WList& w = b->w_resid[l];
    kb_copy_back<T, LY::NU><<<w.nblocks, TPB, 0, b->stream>>>(it(b, w), w.n, (const InstDev<T>*)b->D, b->ctl, l);
    FMB_LAUNCHED();
    return FM_OK;
  }

  // Per level, time every variant of the fused sweep over all instances
  // (one warm-up and TUNE_REPS timed launches, CUDA events) and keep the
  // fastest; a later variant replaces the choice only if it is 2% faster.
  static int autotune(fm_batch* b) {
    for (int l = 0; l < MAXLEV; ++l) b->rbv[l] = 0;
    const char* fixed = getenv("FM_RB_VARIANT");
    if (fixed && fixed[0]) {
      const int v = atoi(fixed);
      for (int l = 0; l < MAXLEV; ++l) b->rbv[l] = (v >= 0 && v < RB_NVAR) ? v : 0;
      return FM_OK;
    }
    kb_set_active<<<(b->count + 255) / 256, 256, 0, b->stream>>>(b->ctl, b->count);
    FMB_LAUNCHED();
    cudaEvent_t e0, e1;
    FMB_CUDA(cudaEventCreate(&e0));
    FMB_CUDA(cudaEventCreate(&e1));
    int rc = FM_OK;
    for (int l = 0; l < b->maxdepth && rc == FM_OK; ++l) {
      float best = 1e30f;
      for (int v = 0; v < RB_TMA0 && rc == FM_OK; ++v) {  // 27..29 repeat 24, 0, 26 here
        rc = launch_variant(b, v, l);
        if (rc == FM_EINVAL) {  // does not fit in shared memory: skip
          rc = FM_OK;
          continue;
        }
        if (rc) break;
        if (cudaEventRecord(e0, b->stream) != cudaSuccess) { rc = FM_ECUDA; break; }
        for (int k = 0; k < TUNE_REPS && rc == FM_OK; ++k) rc = launch_variant(b, v, l);
        if (rc) break;
        float ms = 0.f;
        if (cudaEventRecord(e1, b->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rc = FM_ECUDA;
          break;
        }
        ms /= sweeps_per_launch(v);  // compared per sweep
        b->rbt[l][v] = ms / TUNE_REPS;
        if (ms < best * 0.98f) {  // a later variant must be clearly faster
          best = ms;
          b->rbv[l] = v;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    return rc;
  }

  static int vcycle(fm_batch* b) {
    const InstDev<T>* D = (const InstDev<T>*)b->D;
    const Phys<T>* P = (const Phys<T>*)b->P;
    cudaStream_t s = b->stream;
    // in_r[l]: the correction of level l is in its r buffer (between the pre-
    // and the post-smoothing after an odd number of fused launches)
    int in_r[MAXLEV] = {0};
    for (int l = 0; l < b->maxdepth; ++l) {
      int rc = smooth(b, l, b->prm.nu1, &in_r[l]);
      if (rc) return rc;
      const WList& wq = b->w_rr[l];
      if (wq.n == 0) continue;
      kb_resid_restrict2<T, KIND><<<wq.nblocks, TPB, 0, s>>>(it(b, wq), wq.n, D, P, b->ctl, l, in_r[l]);
      FMB_LAUNCHED();
    }
    if (b->small_global)
      kb_small_global<T, KIND><<<b->count, SMALL_TPB, 0, s>>>(D, P, b->ctl, b->prm.nu1, b->prm.nu2, b->prm.ncoarse);
    else
      kb_small<T, KIND><<<b->count, SMALL_TPB, b->small_smem, s>>>(D, P, b->ctl, b->prm.nu1, b->prm.nu2,
                                                                    b->prm.ncoarse);
    FMB_LAUNCHED();
    for (int l = b->maxdepth - 1; l >= 0; --l) {
      const WList& wp = b->w_prolong[l];
      if (wp.n == 0) continue;
      kb_prolong<T, LY::NU><<<wp.nblocks, TPB, 0, s>>>(it(b, wp), wp.n, D, P, b->ctl, l, in_r[l]);
      FMB_LAUNCHED();
      int rc = smooth(b, l, b->prm.nu2, &in_r[l]);
      if (rc) return rc;
      if (in_r[l]) {
        rc = copy_back(b, l);
        if (rc) return rc;
      }
    }
    return FM_OK;
  }

  static int resid_norm(fm_batch* b, int in_body, cudaGraphConditionalHandle hdl) {
    const InstDev<T>* D = (const InstDev<T>*)b->D;
    const WList& w = b->w_resid64;
    kb_resid64<T, KIND><<<w.nblocks, TPB, 0, b->stream>>>(it(b, w), w.n, D, b->P64, b->K64, b->ctl, in_body);
    FMB_LAUNCHED();
    kb_norm<T, LY::NU><<<b->count, TPB, 0, b->stream>>>(D, b->ctl, b->prm.tol, b->prm.max_cycles, in_body);
    FMB_LAUNCHED();
    kb_condition<<<1, 256, 0, b->stream>>>(b->ctl, b->count, hdl);
    FMB_LAUNCHED();
    return FM_OK;
  }

  static int pre(fm_batch* b, cudaGraphConditionalHandle hdl) {
    const InstDev<T>* D = (const InstDev<T>*)b->D;
    cudaStream_t s = b->stream;
    if (KIND == KCDFT) {
      for (int i = 0; i < b->count; ++i) {
        fm_state* st = b->inst[i];
        st->stream = s;
        const long long l0 = st->launches;
        const int rc = fft_convolve(st, st->rho, st->conv);
        b->launches += st->launches - l0;
        st->stream = b->user_stream;
        if (rc) return rc;
      }
    }
    kb_set_active<<<(b->count + 255) / 256, 256, 0, s>>>(b->ctl, b->count);  // clears the flags
    FMB_LAUNCHED();
    const WList& w = b->w_fine;
    kb_prepare<T, KIND><<<w.nblocks, TPB, 0, s>>>(it(b, w), w.n, D, b->P64, b->K64);
    FMB_LAUNCHED();
    if (KIND == KPFC) {
      kb_prepare_mu<T><<<w.nblocks, TPB, 0, s>>>(it(b, w), w.n, D, b->P64, b->K64);
      FMB_LAUNCHED();
    }
    const WList& wi = b->w_inject;
    if (wi.n) {
      kb_inject<T><<<wi.nblocks, TPB, 0, s>>>(it(b, wi), wi.n, D, b->ctl, 0, 0);
      FMB_LAUNCHED();
    }
    return resid_norm(b, 0, hdl);
  }

  static int body(fm_batch* b, cudaGraphConditionalHandle hdl) {
    const InstDev<T>* D = (const InstDev<T>*)b->D;
    const WList& wi = b->w_inject;
    if (wi.n) {
      kb_inject<T><<<wi.nblocks, TPB, 0, b->stream>>>(it(b, wi), wi.n, D, b->ctl, 1, 1);
      FMB_LAUNCHED();
    }
    int rc = vcycle(b);
    if (rc) return rc;
    const WList& w = b->w_fine;
    kb_update64<T, LY::NU><<<w.nblocks, TPB, 0, b->stream>>>(it(b, w), w.n, D, b->ctl, b->prm.delta);
    FMB_LAUNCHED();
    return resid_norm(b, 1, hdl);
  }

  static int post(fm_batch* b) {
    const InstDev<T>* D = (const InstDev<T>*)b->D;
    const WList& w = b->w_fine;
    kb_closure<T><<<w.nblocks, TPB, 0, b->stream>>>(it(b, w), w.n, D, b->P64, b->K64, b->ctl);
    FMB_LAUNCHED();
    kb_commit<T><<<w.nblocks, TPB, 0, b->stream>>>(it(b, w), w.n, D, b->ctl);
    FMB_LAUNCHED();
    FMB_CUDA(cudaMemcpyAsync(b->hctl, b->ctl, sizeof(Ctl) * b->count, cudaMemcpyDeviceToHost, b->stream));
    return FM_OK;
  }

  static int build_graph(fm_batch* b) {
    cudaStream_t saved = b->stream;
    cudaStream_t s0 = b->cap[0], s1 = b->cap[1];
    b->stream = s0;
    int rc = FM_OK;
    cudaGraph_t g = nullptr;
    const long long l0 = b->launches;
    do {
      if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = FM_ECUDA; break; }
      cudaStreamCaptureStatus cs;
      cudaGraph_t cg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      if (cudaStreamGetCaptureInfo(s0, &cs, nullptr, &cg, nullptr, nullptr, nullptr) != cudaSuccess) { rc = FM_ECUDA; break; }
      cudaGraphConditionalHandle hdl;
      if (cudaGraphConditionalHandleCreate(&hdl, cg, 0, cudaGraphCondAssignDefault) != cudaSuccess) { rc = FM_ECUDA; break; }
      rc = pre(b, hdl);
      if (rc) break;
      b->cnt_pre = b->launches - l0;
      if (cudaStreamGetCaptureInfo(s0, &cs, nullptr, &cg, &deps, nullptr, &nd) != cudaSuccess) { rc = FM_ECUDA; break; }
      cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
      cp.conditional.handle = hdl;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t wnode;
      if (cudaGraphAddNode(&wnode, cg, deps, nullptr, nd, &cp) != cudaSuccess) { rc = FM_ECUDA; break; }
      cudaGraph_t bodyg = cp.conditional.phGraph_out[0];
      if (cudaStreamUpdateCaptureDependencies(s0, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess) { rc = FM_ECUDA; break; }
      b->stream = s1;
      if (cudaStreamBeginCaptureToGraph(s1, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { rc = FM_ECUDA; break; }
      const long long l1 = b->launches;
      rc = body(b, hdl);
      b->cnt_body = b->launches - l1;
      cudaGraph_t bo = nullptr;
      if (cudaStreamEndCapture(s1, &bo) != cudaSuccess && rc == FM_OK) rc = FM_ECUDA;
      if (rc) break;
      b->stream = s0;
      const long long l2 = b->launches;
      rc = post(b);
      b->cnt_post = b->launches - l2;
    } while (0);
    b->stream = s0;
    if (cudaStreamEndCapture(s0, &g) != cudaSuccess && rc == FM_OK) rc = FM_ECUDA;
    b->stream = saved;
    b->launches = l0;
    if (rc) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(g);
      return FM_ECUDA;
    }
    b->graph = g;
    return FM_OK;
  }

  static int setup(fm_batch* b) {
    std::vector<InstDev<T>> H(b->count);
    b->small_smem = 0;
    b->small_global = false;
    build_desc(b, H);
    build_lists(b);
    const size_t szD = sizeof(InstDev<T>) * b->count;
    const size_t szP = sizeof(Phys<T>) * b->count;
    const size_t szP64 = sizeof(Phys<double>) * b->count;
    const size_t szK64 = sizeof(Step64) * b->count;
    const size_t szC = sizeof(Ctl) * b->count;
    const size_t szI = sizeof(WorkItem) * (b->hitems.size() + 1);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t total = al(szD) + al(szP) + al(szP64) + al(szK64) + al(szC) + al(szI);
    FMB_CUDA(cudaMalloc(&b->dev, total));
    char* p = (char*)b->dev;
    b->D = p; p += al(szD);
    b->P = p; p += al(szP);
    b->P64 = (Phys<double>*)p; p += al(szP64);
    b->K64 = (Step64*)p; p += al(szK64);
    b->ctl = (Ctl*)p; p += al(szC);
    b->items = (WorkItem*)p;
    // the non-positive-density flag of an instance lives in the batch's
    // control block, not in the instance's own
    for (int i = 0; i < b->count; ++i) H[i].F.nonpos = KIND == KCDFT ? &b->ctl[i].nonpos : nullptr;
    FMB_CUDA(cudaMemcpy(b->D, H.data(), szD, cudaMemcpyHostToDevice));
    if (!b->hitems.empty())
      FMB_CUDA(cudaMemcpy(b->items, b->hitems.data(), sizeof(WorkItem) * b->hitems.size(), cudaMemcpyHostToDevice));
    FMB_CUDA(cudaMemset(b->ctl, 0, szC));
    FMB_CUDA(cudaMallocHost(&b->hP, szP));
    FMB_CUDA(cudaMallocHost((void**)&b->hP64, szP64));
    FMB_CUDA(cudaMallocHost((void**)&b->hK64, szK64));
    FMB_CUDA(cudaMallocHost((void**)&b->hctl, szC));
    if (b->small_smem > (size_t)SMALL_SMEM_MAX) b->small_global = true;
    if (!b->small_global)
      FMB_CUDA(cudaFuncSetAttribute(kb_small<T, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)SMALL_SMEM_MAX));
    return autotune(b);
    return FM_OK;
  }

  // Time `iters` finest-level launches of fused-sweep variant v over all
  // instances (CUDA events on the batch stream); the corrections they write
  // are scratch that the next step resets.
  static int time_smoother(fm_batch* b, int v, int iters, double* ms) {
    kb_set_active<<<(b->count + 255) / 256, 256, 0, b->stream>>>(b->ctl, b->count);
    FMB_LAUNCHED();
    cudaEvent_t e0, e1;
    FMB_CUDA(cudaEventCreate(&e0));
    FMB_CUDA(cudaEventCreate(&e1));
    int rc = launch_variant(b, v, 0);  // warm-up
    if (rc == FM_OK && cudaEventRecord(e0, b->stream) != cudaSuccess) rc = FM_ECUDA;
    for (int k = 0; k < iters && rc == FM_OK; ++k) rc = launch_variant(b, v, 0);
    if (rc == FM_OK && cudaEventRecord(e1, b->stream) != cudaSuccess) rc = FM_ECUDA;
    if (rc == FM_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = FM_ECUDA;
    float t = 0.f;
    if (rc == FM_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) rc = FM_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    *ms = (double)t / iters;
    return rc;
  }

  static int step(fm_batch* b, const double* dt) {
    Phys<T>* hp = (Phys<T>*)b->hP;
    for (int i = 0; i < b->count; ++i) {
      b->inst[i]->dt = dt[i];
      hp[i] = make_phys<T>(b->inst[i]);
      b->hP64[i] = make_phys<double>(b->inst[i]);
      b->hK64[i] = make_step64(b->hP64[i], 1.0 / b->inst[i]->lv[0].h);
    }
    FMB_CUDA(cudaMemcpyAsync(b->P, hp, sizeof(Phys<T>) * b->count, cudaMemcpyHostToDevice, b->stream));
    FMB_CUDA(cudaMemcpyAsync(b->P64, b->hP64, sizeof(Phys<double>) * b->count, cudaMemcpyHostToDevice, b->stream));
    FMB_CUDA(cudaMemcpyAsync(b->K64, b->hK64, sizeof(Step64) * b->count, cudaMemcpyHostToDevice, b->stream));
    if (!b->gexec) {
      const int rc = build_graph(b);
      if (rc) return rc;
    }
    FMB_CUDA(cudaGraphLaunch(b->gexec, b->stream));
    FMB_CUDA(cudaStreamSynchronize(b->stream));
    long long maxc = 0;
    for (int i = 0; i < b->count; ++i)
      if (b->hctl[i].cycles > maxc) maxc = b->hctl[i].cycles;
    b->launches += b->cnt_pre + maxc * b->cnt_body + b->cnt_post;
    return FM_OK;
  }
};

template <typename T>
static int batch_dispatch_setup(fm_batch* b) {
  return b->kind == FM_PFC ? Batch<T, KPFC>::setup(b) : Batch<T, KCDFT>::setup(b);
}
template <typename T>
static int batch_dispatch_step(fm_batch* b, const double* dt) {
  return b->kind == FM_PFC ? Batch<T, KPFC>::step(b, dt) : Batch<T, KCDFT>::step(b, dt);
}

}  // namespace fm

extern "C" {

void fm_destroy_batch(fm_batch* b) {
  if (!b) return;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (int i = 0; i < 2; ++i)
    if (b->cap[i]) cudaStreamDestroy(b->cap[i]);
  if (b->dev) cudaFree(b->dev);
  if (b->hP) cudaFreeHost(b->hP);
  if (b->hP64) cudaFreeHost(b->hP64);
  if (b->hK64) cudaFreeHost(b->hK64);
  if (b->hctl) cudaFreeHost(b->hctl);
  if (b->inst) {
    for (int i = 0; i < b->count; ++i) fm_destroy(b->inst[i]);
    delete[] b->inst;
  }
  delete b;
}

int fm_create_batch(int count, const fm_grid* grids, const fm_params* prm, const fm_functional* fn,
                    fm_batch** out) {
  if (!out || !grids || !prm || !fn || count < 1 || count > 4096) return FM_EINVAL;
  *out = nullptr;
  if (prm->model != FM_HYDRO || prm->walls != FM_WALLS_NONE || prm->init != FM_INIT_PREVIOUS)
    return FM_EINVAL;  // periodic hydrodynamic, each step from its previous time level
  for (int i = 0; i < count; ++i)
    if (grids[i].dim != 2) return FM_EINVAL;  // batched ensembles are 2-D
  fm_batch* b = new (std::nothrow) fm_batch();
  if (!b) return FM_ENOMEM;
  b->count = count;
  b->kind = fn->kind;
  b->prm = *prm;
  b->fn = *fn;
  b->stream = 0;
  b->inst = new (std::nothrow) fm_state*[count]();
  if (!b->inst) {
    delete b;
    return FM_ENOMEM;
  }
  // the batch runs its coarse levels in the cycle's precision (its own
  // per-instance kernels): no float64 copies of them in the instances
  fm_params iprm = *prm;
  if (iprm.coarse_precision != FM_FP64 && iprm.coarse_precision != FM_MIXED) {
    fm_destroy_batch(b);
    return FM_EINVAL;
  }
  iprm.coarse_precision = FM_MIXED;
  for (int i = 0; i < count; ++i) {
    const int rc = fm_create(&grids[i], &iprm, fn, &b->inst[i]);
    if (rc) {
      fm_destroy_batch(b);
      return rc;
    }
  }
  if (cudaStreamCreateWithFlags(&b->cap[0], cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap[1], cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    fm_destroy_batch(b);
    return FM_ECUDA;
  }
  const int rc = prm->precision == FM_MIXED ? batch_dispatch_setup<float>(b) : batch_dispatch_setup<double>(b);
  if (rc) {
    fm_destroy_batch(b);
    return rc;
  }
  *out = b;
  return FM_OK;
}

int fm_batch_set_stream(fm_batch* b, void* stream) {
  if (!b) return FM_EINVAL;
  b->stream = (cudaStream_t)stream;
  b->user_stream = (cudaStream_t)stream;
  for (int i = 0; i < b->count; ++i) fm_set_stream(b->inst[i], stream);
  return FM_OK;
}

fm_state* fm_batch_instance(fm_batch* b, int i) {
  if (!b || i < 0 || i >= b->count) return nullptr;
  return b->inst[i];
}

int fm_step_batch(fm_batch* b, const double* dt, fm_step_info* info) {
  if (!b || !dt) return FM_EINVAL;
  for (int i = 0; i < b->count; ++i)
    if (!(dt[i] > 0.0)) return FM_EINVAL;
  const int rc = b->prm.precision == FM_MIXED ? batch_dispatch_step<float>(b, dt) : batch_dispatch_step<double>(b, dt);
  if (rc) return rc;
  int status = FM_OK;
  for (int i = 0; i < b->count; ++i) {
    if (info) {
      info[i].cycles = b->hctl[i].cycles;
      info[i].res0 = b->hctl[i].norm0;
      info[i].res = b->hctl[i].norm;
    }
    if (b->hctl[i].status != FM_OK && status == FM_OK) status = b->hctl[i].status;
  }
  return status;
}

long long fm_batch_launches(const fm_batch* b) { return b ? b->launches : -1; }

int fm_batch_tuning(const fm_batch* b, int level, int* variant, float* ms_per_variant) {
  if (!b || level < 0 || level >= MAXLEV) return FM_EINVAL;
  if (variant) *variant = b->rbv[level];
  if (ms_per_variant)
    for (int v = 0; v < RB_NVAR; ++v) ms_per_variant[v] = b->rbt[level][v];
  return FM_OK;
}

static int batch_time_variant(fm_batch* b, int variant, int iters, double* ms_per_launch, long long* points) {
  if (!b || iters < 1 || !ms_per_launch) return FM_EINVAL;
  if (b->maxdepth < 1) return FM_EINVAL;  // no instance has a multi-kernel finest level
  const int v = variant < 0 ? b->rbv[0] : variant;
  if (v >= RB_NVAR) return FM_EINVAL;
  long long np = 0;
  for (int i = 0; i < b->count; ++i)
    if (b->inst[i]->small_from > 0) np += b->inst[i]->lv[0].g.N;
  if (points) *points = np;
  if (b->prm.precision == FM_MIXED)
    return b->kind == FM_PFC ? Batch<float, KPFC>::time_smoother(b, v, iters, ms_per_launch)
                             : Batch<float, KCDFT>::time_smoother(b, v, iters, ms_per_launch);
  return b->kind == FM_PFC ? Batch<double, KPFC>::time_smoother(b, v, iters, ms_per_launch)
                           : Batch<double, KCDFT>::time_smoother(b, v, iters, ms_per_launch);
}

int fm_batch_time_smoother(fm_batch* b, int iters, double* ms_per_launch, long long* points) {
  return batch_time_variant(b, -1, iters, ms_per_launch, points);
}

int fm_batch_time_sweep_variant(fm_batch* b, int variant, int iters, double* ms_per_launch, long long* points) {
  if (variant < 0) return FM_EINVAL;
  return batch_time_variant(b, variant, iters, ms_per_launch, points);
}

}  // extern "C"
