// 2-D red-black sweeps of one level in one cooperative launch (App. G.1-G.3
// point block, red-black ordering): the red and the black passes over the
// whole level, in place, separated by a grid-wide barrier instead of kernel
// boundaries, so a level's pre- or post-smoothing is one launch with no halo
// recomputation.  Used by the single-instance solver (2-D variant 34).
#pragma once

#include "fm_device.cuh"

namespace fm {

// Accessor of the point update over the level in global memory.  The
// correction is read through L2 only (ld.global.cg): other blocks rewrite it
// between passes and an SM's L1 is not kept coherent with their stores.  The
// coefficients, right-hand side and omega do not change during the launch.
template <typename T>
struct CoopAcc {
  const Lvl<T>& L;
  __device__ __forceinline__ T e(int q, int i) const { return __ldcg(L.e[q] + i); }
  __device__ __forceinline__ void set_e(int q, int i, T v) const { __stcg(L.e[q] + i, v); }
  __device__ __forceinline__ T rk(int i) const { return __ldg(L.rk + i); }
  __device__ __forceinline__ T cr(int i) const { return __ldg(L.cr + i); }
  __device__ __forceinline__ T cv(int d, int i) const { return __ldg(L.cv[d] + i); }
  __device__ __forceinline__ T f(int q, int i) const { return __ldg(L.f[q] + i); }
  __device__ __forceinline__ T om(int d, int i) const { return __ldg(L.om[d] + i); }
};

// Grid-wide barrier number k (1, 2, ...) of a launch whose blocks are all
// resident (cooperative launch): every block adds one arrival to bar[0] and
// waits until it counts k * gridDim.x.  The wait gives up after limit_ns:
// the block then sets *fault and the call returns false in all its threads.
// The fences order each block's stores of the pass before its arrival and
// the other blocks' stores before its next pass.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned k, int* fault, unsigned long long limit_ns) {
  __syncthreads();
  bool ok = true;
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned target = k * gridDim.x;
    const volatile unsigned* vb = bar;
    if (*vb < target) {
      const unsigned long long t0 = global_ns();
      while (*vb < target) {
        if (global_ns() - t0 > limit_ns) {
          atomicExch(fault, 1);
          ok = false;
          break;
        }
      }
    }
    __threadfence();
  }
  return __syncthreads_and(ok) != 0;
}

// The last block to leave resets the barrier for the next launch (launches
// on the stream follow one another, so the next one starts from zero).
__device__ __forceinline__ void grid_barrier_leave(unsigned* bar) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(bar + 1, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      atomicExch(bar + 1, 0u);
    }
  }
}

// nsweeps red-black sweeps of level L in place: 2 nsweeps passes (red points,
// i + j even, first), each a grid-stride loop over the points of its colour,
// with a grid barrier between passes.  A red pass reads black values only
// and a black pass red values only, all final after the barrier, so the
// result is that of nsweeps red and black launch pairs.  A block whose
// barrier wait runs out returns without leaving (*fault is set; the step
// reports FM_ETIMEOUT).
template <typename T, int KIND>
__global__ void __launch_bounds__(TPB) k_smooth_coop(const __grid_constant__ Lvl<T> L, Phys<T> P, int nsweeps,
                                                     unsigned* bar, int* fault) {
  const PtK<T> K = make_ptk<T, 2>(P, L.h);
  const CoopAcc<T> a{L};
  const int half = L.g.N >> 1;
  const int stride = gridDim.x * blockDim.x;
  const int npass = 2 * nsweeps;
  for (int pass = 0; pass < npass; ++pass) {
    const int color = pass & 1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < half; t += stride) {
      int i, j, k;
      colour_point(t, color, L.g, i, j, k);
      const Nb n = neighbours(i, j, k, L.g);
      smooth_point_a<T, KIND, 2>(a, P, K, n, n.c);
    }
    if (pass + 1 < npass && !grid_barrier(bar, (unsigned)(pass + 1), fault, TMA_WAIT_NS)) return;
  }
  grid_barrier_leave(bar);
}

}  // namespace fm
