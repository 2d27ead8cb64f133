// 3-D fused red-black sweep, z-marching form (App. G.1-G.3 point block,
// red-black ordering), used by the single-instance solver on 3-D levels.
#pragma once

#include "fm_device.cuh"

namespace fm {

// A block owns an xy tile of 32 x TY points, tile (i, j) starting at
// x0 = 32 i + 2, y0 = TY j (the tiling is shifted by two columns so that the
// staged rows, columns x0 - 2 .. x0 + 33, start on a 16-byte boundary), and a
// range of its planes [z0, z1).  It marches up the planes one per step.  Step
// p updates, in one phase,
//   * the red points of plane p + 2 on the tile and on the ring around it
//     that the tile's black points see (rows y0 - 1 and y0 + TY over the
//     tile's columns; columns x0 - 1 and x0 + 32 over its rows), and
//   * the black points of plane p on the tile,
// then plane p - 1, final since step p - 1, is written out.  Red updates read
// black values from before the sweep; black updates read the new red values
// of planes p - 1 .. p + 1, all computed by steps p - 3 .. p - 1 of the same
// block (the ring's red points are computed again by the blocks that own
// them, from the same values, so they are identical).  The correction is
// read from one buffer and written to the other, so every staged value is
// from before the sweep whatever the block schedule, and the result is
// exactly one red-black sweep.
//
// The arrays the point update reads at neighbours -- e (NU), rho^k, the
// coefficient velocity (3) and, for CDFT, the coefficient density -- are
// staged plane by plane into a ring of 5 + D slots (planes p - 1 .. p + 3 + D
// are live in step p) by 16-byte cp.async chunks: thread t below SR * SW / V
// owns one chunk position of the plane and copies it for every array.  The
// copies of plane p + 3 + D are issued at the start of step p, and at its end
// the step waits for those of plane p + 4 (D = 1: issued by this step; D = 2:
// by the step before).  (Staging each row by one bulk copy through the tensor
// memory accelerator, 120 copies of 144 bytes per plane, measured three times
// slower: the per-copy cost of the unit, not the bytes, set the pace.)  The
// right-hand side, omega^k and (PFC) the coefficient density are read only
// at the point itself: each thread loads them into registers one step ahead.
//
// Warps of a block (TY + 2): TY / 2 red warps on the tile (two rows each,
// sixteen red points a row: the rows' opposite parities put the two half
// warps on opposite shared-memory banks), one red warp on the two ring rows,
// one on the two ring columns (TY lanes), TY / 2 black warps on the tile.
// Every active lane does one point update per step.
template <int TY>
struct ZmGeom {
  static constexpr int TX = 32;
  static constexpr int SW = TX + 4;  // staged columns x0 - 2 .. x0 + 33
  static constexpr int SR = TY + 4;  // staged rows y0 - 2 .. y0 + TY + 1
  static constexpr int PS = SW * SR;  // values of one array in one plane
  // ring slots and copy distance D = NSLOT - 5 (planes issued D steps before
  // the step that first reads them).  Six slots, D = 1: a seventh slot for
  // D = 2 on 32 x 16 tiles (202 KB of shared memory) measured slower, 0.093
  // against 0.072 ms per sweep at 128^3 -- it leaves too little L1 for the
  // point values that a red and a black point of one sector load in turn.
  static constexpr int NSLOT = 6;
  static constexpr int D = NSLOT - 5;
  static constexpr int WARPS = TY + 2;
  static constexpr int THREADS = 32 * WARPS;
};

template <int KIND>
__host__ __device__ constexpr int zm_arrays() {
  return Layout<KIND, 3>::NU + 4 + (KIND == KCDFT ? 1 : 0);  // e, rk, cv0..2 (, cr)
}
template <typename T, int KIND, int TY>
__host__ __device__ constexpr size_t zm_smem_bytes() {
  return (size_t)ZmGeom<TY>::NSLOT * zm_arrays<KIND>() * ZmGeom<TY>::PS * sizeof(T) + 128;  // + alignment
}
// Resident blocks per SM the float32 kernels are compiled for.
template <typename T>
__host__ __device__ constexpr int zm_minb(int ty) { return (sizeof(T) == 4 && ty == 8) ? 2 : 1; }

// Values of one point read only at that point.
template <typename T, int KIND>
struct ZmPt {
  T fv[Layout<KIND, 3>::NU];
  T om[3];
  T crv;
};

template <typename T, int KIND>
__device__ __forceinline__ void zm_load_pt(const Lvl<T>& G, int gi, ZmPt<T, KIND>& p) {
#pragma unroll
  for (int q = 0; q < Layout<KIND, 3>::NU; ++q) p.fv[q] = G.f[q][gi];
#pragma unroll
  for (int d = 0; d < 3; ++d) p.om[d] = G.om[d][gi];
  p.crv = KIND == KPFC ? G.cr[gi] : T(0);
}

// Accessor of the point update over the plane ring (index = slot base +
// staged point, array a at offset a * PS) and one point's register values.
template <typename T, int KIND, int PS>
struct ZmAcc {
  static constexpr int NU = Layout<KIND, 3>::NU;
  T* sm;
  const ZmPt<T, KIND>& p;
  __device__ __forceinline__ T e(int q, int i) const { return sm[i + q * PS]; }
  __device__ __forceinline__ void set_e(int q, int i, T v) const { sm[i + q * PS] = v; }
  __device__ __forceinline__ T rk(int i) const { return sm[i + NU * PS]; }
  __device__ __forceinline__ T cv(int d, int i) const { return sm[i + (NU + 1 + d) * PS]; }
  __device__ __forceinline__ T cr(int i) const {
    if constexpr (KIND == KCDFT) return sm[i + (NU + 4) * PS];
    else return p.crv;  // the PFC update reads the coefficient density at the point only
  }
  __device__ __forceinline__ T f(int q, int) const { return p.fv[q]; }
  __device__ __forceinline__ T om(int d, int) const { return p.om[d]; }
};

// The point this lane updates at plane z (unwrapped) in its warp's role
// (see above): tile coordinates (tx, ty), tx = -1 .. 32, ty = -1 .. TY.
// Red points have x + y + z even; x0 is even and every grid size is even, so
// parities of unwrapped coordinates are those of the wrapped ones.
template <int TY>
__device__ __forceinline__ bool zm_point(int warp, int lane, int y0, int z, int& tx, int& ty) {
  if (warp < TY / 2) {  // red, tile rows
    ty = 2 * warp + (lane >> 4);
    tx = 2 * (lane & 15) + ((y0 + ty + z) & 1);
    return true;
  }
  if (warp == TY / 2) {  // red, ring rows
    ty = lane < 16 ? -1 : TY;
    tx = 2 * (lane & 15) + ((y0 + ty + z) & 1);
    return true;
  }
  if (warp == TY / 2 + 1) {  // red, ring columns
    if (lane >= TY) return false;
    ty = lane;
    tx = ((y0 + ty + z) & 1) ? -1 : 32;
    return true;
  }
  ty = 2 * (warp - TY / 2 - 2) + (lane >> 4);  // black, tile rows
  tx = 2 * (lane & 15) + ((y0 + ty + z + 1) & 1);
  return true;
}

// One sweep of the level.  Every tile is cut into z-chunks, nchunks of them
// for tiles 0 .. nlong - 1 and nchunks + 1 for the others (so that the blocks
// fill the resident slots; the longer chunks come first, so that the blocks
// the device runs side by side on one multiprocessor tend to pair a long
// chunk with a short one), one block per chunk.  The blocks of all tiles start
// together at the chunk boundaries and march up the planes side by side, so
// the halos they share are read from L2.  Reads the correction from G.e
// (dir = 0) or G.r (dir = 1) and writes it to the other.
template <typename T, int KIND, int TY>
__global__ void __launch_bounds__(ZmGeom<TY>::THREADS, zm_minb<T>(TY))
    k_smooth_zm3(const __grid_constant__ Lvl<T> G, Phys<T> P, int dir, int nchunks, int nlong) {
  using Gm = ZmGeom<TY>;
  constexpr int NU = Layout<KIND, 3>::NU;
  constexpr int NA = zm_arrays<KIND>();
  constexpr int SW = Gm::SW, PS = Gm::PS, NSLOT = Gm::NSLOT;
  constexpr int SS = NA * PS;  // slot stride
  constexpr int V = 16 / sizeof(T);
  constexpr int CPR = SW / V;           // 16-byte chunks per staged row
  constexpr int NPOS = Gm::SR * CPR;    // chunk positions of a plane (each over all NA arrays)
  static_assert(NPOS <= Gm::THREADS, "one staging thread per chunk position");
  const unsigned s0 = smem_u32(fm_dyn_smem);
  T* ring = reinterpret_cast<T*>(fm_dyn_smem + (((s0 + 127u) & ~127u) - s0));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool red = warp <= TY / 2 + 1;
  const int nx = G.g.nx, ny = G.g.ny, nz = G.g.nz;
  const int plane = nx * ny;
  const int nbx = nx / Gm::TX, ntile = nbx * (ny / TY);
  // blocks [0, nlong * nchunks): tiles 0 .. nlong - 1 in nchunks z-chunks;
  // the rest: the other tiles in nchunks + 1 z-chunks
  int tile, chunk, nch;
  if ((int)blockIdx.x < nlong * nchunks) {
    tile = blockIdx.x % nlong;
    chunk = blockIdx.x / nlong;
    nch = nchunks;
  } else {
    const int b = blockIdx.x - nlong * nchunks, nshort = ntile - nlong;
    tile = nlong + b % nshort;
    chunk = b / nshort;
    nch = nchunks + 1;
  }
  const int z0 = (int)((long long)chunk * nz / nch), z1 = (int)((long long)(chunk + 1) * nz / nch);
  const int x0 = (tile % nbx) * Gm::TX + 2, y0 = (tile / nbx) * TY;
  T* const* dst = dir ? G.e : G.r;
  const PtK<T> K = make_ptk<T, 3>(P, G.h);
  // staged planes z0 - 2 .. z1 + 1; plane z lives in slot (z - z0 + 2) % NSLOT
  auto slot_base = [&](int z) { return (int)((unsigned)(z - z0 + 2) % (unsigned)NSLOT) * SS; };
  auto next_slot = [&](int b) { return b + SS == NSLOT * SS ? 0 : b + SS; };
  auto wrapz = [&](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
  // this thread's staged chunk position (threads below NPOS), the same in every plane
  const bool stager = tid < NPOS;
  int s_off = 0, g_off = 0;
  if (stager) {
    const int r = tid / CPR, c = tid - r * CPR;
    s_off = r * SW + c * V;
    g_off = wrapi(y0 - 2 + r, ny) * nx + wrapi(x0 - 2 + c * V, nx);
  }
  auto issue = [&](int z) {
    if (!stager) return;
    T* d = ring + slot_base(z) + s_off;
    const int gi = wrapz(z) * plane + g_off;
#pragma unroll
    for (int a = 0; a < NA; ++a) {
      const T* src;
      if (a < NU) src = dir ? G.r[a] : G.e[a];
      else if (a == NU) src = G.rk;
      else if (a < NU + 4) src = G.cv[a - NU - 1];
      else src = G.cr;
      cp_async_16(d + a * PS, src + gi);
    }
  };
  // this lane's point for planes of either parity: staged and global
  // in-plane offsets (zm_point depends on z only through its parity)
  int sxy0 = 0, sxy1 = 0, gxy0 = 0, gxy1 = 0;
  bool has;
  {
    int tx, ty;
    has = zm_point<TY>(warp, lane, y0, 0, tx, ty);
    if (has) {
      sxy0 = (ty + 2) * SW + tx + 2;
      gxy0 = wrapi(y0 + ty, ny) * nx + wrapi(x0 + tx, nx);
      zm_point<TY>(warp, lane, y0, 1, tx, ty);
      sxy1 = (ty + 2) * SW + tx + 2;
      gxy1 = wrapi(y0 + ty, ny) * nx + wrapi(x0 + tx, nx);
    }
  }
  auto sxy = [&](int z) { return (z & 1) ? sxy1 : sxy0; };
  auto gxy = [&](int z) { return (z & 1) ? gxy1 : gxy0; };
  // the plane of this lane's role in step p, or false
  auto role_z = [&](int p, int& z) {
    z = red ? p + 2 : p;
    return has && (red ? (z >= z0 - 1 && z <= z1) : (z >= z0 && z < z1));
  };

  // the first 16 TY threads (red tile warps) write the final planes out, two
  // values a lane: in-plane staged and global offsets of the lane's pair
  // (measured faster than giving it to the black warps)
  const int wb = tid < 16 * TY ? tid : -1;
  int wb_s = 0, wb_g = 0;
  if (wb >= 0) {
    const int ty = wb >> 4, i = wb & 15;
    wb_s = (ty + 2) * SW + 2 + 2 * i;
    wb_g = wrapi(y0 + ty, ny) * nx + wrapi(x0 + 2 * i, nx);
  }
  // step p: issue plane p + 3 + D; write plane p - 1 out; this lane's update
  // with its point values `cur`; load the next step's into `nxt`; wait for
  // plane p + 4 (every step commits one copy group, empty at the end)
  auto step = [&](int p, const ZmPt<T, KIND>& cur, ZmPt<T, KIND>& nxt) {
    // slots of the planes z - 1, z, z + 1 around this warp's role plane z
    // (red: p + 2, black: p)
    const int sbm = slot_base(red ? p + 1 : p - 1);
    const int sbc = next_slot(sbm), sbp = next_slot(sbc);
    if (p + 3 + Gm::D <= z1 + 1) issue(p + 3 + Gm::D);
    cp_async_commit();
    if (p - 1 >= z0 && p - 1 < z1 && wb >= 0) {
      const int si = slot_base(p - 1) + wb_s;
      const int gi = wrapz(p - 1) * plane + wb_g;
#pragma unroll
      for (int q = 0; q < NU; ++q) {
        if constexpr (sizeof(T) == 4) {
          *reinterpret_cast<float2*>(dst[q] + gi) = *reinterpret_cast<const float2*>(ring + si + q * PS);
        } else {
          *reinterpret_cast<double2*>(dst[q] + gi) = *reinterpret_cast<const double2*>(ring + si + q * PS);
        }
      }
    }
    int z;
    if (role_z(p, z)) {
      const ZmAcc<T, KIND, PS> acc{ring, cur};
      const int xy = sxy(z);
      Nb n;
      n.c = sbc + xy;
      n.m[0] = n.c - 1;
      n.p[0] = n.c + 1;
      n.m[1] = n.c - SW;
      n.p[1] = n.c + SW;
      n.m[2] = sbm + xy;
      n.p[2] = sbp + xy;
      smooth_point_a<T, KIND, 3>(acc, P, K, n, 0);
    }
    if (role_z(p + 1, z)) zm_load_pt<T, KIND>(G, wrapz(z) * plane + gxy(z), nxt);
    cp_async_wait_n<Gm::D - 1>();
    __syncthreads();
  };

  // prologue: planes z0 - 2 .. z0 (step z0 - 3 reads them) in one group,
  // then z0 + 1 .. z0 + D - 1 one group each (left in flight)
  for (int z = z0 - 2; z <= z0; ++z) issue(z);
  cp_async_commit();
  for (int z = z0 + 1; z <= z0 + Gm::D - 1; ++z) {
    if (z <= z1 + 1) issue(z);
    cp_async_commit();
  }
  ZmPt<T, KIND> pa, pb;
  {
    int z;
    if (role_z(z0 - 3, z)) zm_load_pt<T, KIND>(G, wrapz(z) * plane + gxy(z), pa);
  }
  cp_async_wait_n<Gm::D - 1>();
  __syncthreads();
  // steps z0 - 3 .. z1, two per iteration (the point values alternate
  // between pa and pb)
#pragma unroll 1
  for (int p = z0 - 3; p <= z1; p += 2) {
    step(p, pa, pb);
    if (p + 1 <= z1) step(p + 1, pb, pa);
  }
}

}  // namespace fm
