// ce_sweep3d.cuh -- the 3D z-sweep fused leapfrog step for sm_103a (device code).
//
// Same arithmetic per site as the generic kernel (ce_generic.cu): with state
// (f_n, w_n) and f'(t_n + dt/2) = w + c f,
//   v = w + c f,  g = f + dt v  (= f_{n+1}),
//   w_out = v + dt (lap g - dV/df(g)),  f_out = g,
// plus the block sums of (g(x+e_d) - g(x))^2 and V(g) that drive a(t)
// (arXiv:0712.0813 Sec. III staggered leapfrog; the paper's ghost columns and
// edge exchange become the periodic index arithmetic of one HBM-resident
// lattice).
//
// Decomposition.  A CTA owns a TX x TY tile of (x, y) and sweeps a chunk of z.
// Each xy plane of f and w (all fields) is brought into shared memory by TMA
// (cp.async.bulk.tensor, one elected thread, mbarrier completion) as a box of
// TY+2 rows x TX columns: the tile plus one halo row on each side in y.  At the
// y edges of the lattice the box is split so that the wrapped halo row lands in
// its place (a TY+1-row box plus a 1-row box); tensor-map boxes never leave the
// array, so no zero-filled element is ever used.  The z-neighbours of a site
// are its own column in the previous and next planes and stay in registers;
// the x-neighbours come from the adjacent lane (warp shuffle, a warp spans one
// row of TX = 32 * VX sites, VX = 16 B / sizeof(T) per thread) except at the
// two row ends, whose wrapped halo values are read with plain loads two planes
// ahead.  A ring of NST stages keeps NST - 2 planes in flight while one plane
// is computed.  HBM traffic per site and step is the ideal read f, w + write
// f, w per field; halo rows are re-read from L2 by the neighbouring tile.
//
// Every wait on an mbarrier is bounded: on expiry the kernel latches
// CE_ETIMEOUT in the device status word, waits (bounded) for its own copies
// still in flight and leaves the sweep, still taking part in the end-of-step
// reduction so the launch completes.
#pragma once

#include <cuda.h>

#include <cstdint>

#include "ce_device.cuh"
#include "ce_internal.h"
#include "ce_tma.cuh"

namespace ce {
namespace sweep {

// Kernel variants (rows per tile TY, pipeline stages NST) compiled into the
// library; the plan picks one (an autotuner may pick it instead).
struct Variant {
  int ty;
  int stages;
};
constexpr Variant kVariants[] = {{8, 4}, {8, 5}, {16, 3}, {16, 4}, {4, 4}, {4, 5}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

// Bytes of one x-halo column buffer (TY rows of 16 bytes), padded to the
// 128-byte alignment every TMA destination needs.
__host__ __device__ constexpr size_t halo_bytes(int ty) { return ((size_t)ty * 16 + 127) / 128 * 128; }

template <typename T>
constexpr size_t smem_bytes(int nf, int ty, int stages) {
  return (size_t)stages * nf * 2 * ((ty + 2) * (32 * (16 / sizeof(T))) * sizeof(T) + 2 * halo_bytes(ty)) +
         3 * stages * sizeof(uint64_t) + 128;
}

// Resident CTAs per SM the kernel is compiled for (register budget): as many
// as shared memory admits, up to 2 for 8-row tiles and 4 for 4-row tiles.
template <typename T, int NF, int TY, int NST>
constexpr int min_blocks() {
  constexpr size_t by_smem = (220 * 1024) / smem_bytes<T>(NF, TY, NST);
  constexpr int cap = TY <= 4 ? 4 : (TY <= 8 ? 2 : 1);
  return by_smem < 1 ? 1 : (by_smem < (size_t)cap ? (int)by_smem : cap);
}



// VX consecutive values of one row: one 16-byte shared-memory access.
template <typename T, int VX>
__device__ __forceinline__ void lds16(const T* p, T (&o)[VX]) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    const double2 v = *reinterpret_cast<const double2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
}

// VX consecutive values of one row: one 16-byte shared-memory store.
template <typename T, int VX>
__device__ __forceinline__ void sts16(T* p, const T (&o)[VX]) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  } else {
    *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
  }
}

// 16-byte streaming store to HBM (the next step reads it back from HBM anyway).
template <typename T, int VX>
__device__ __forceinline__ void stg16(T* p, const T (&o)[VX]) {
  if constexpr (sizeof(T) == 4) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(o[0], o[1], o[2], o[3]));
  } else {
    __stcs(reinterpret_cast<double2*>(p), make_double2(o[0], o[1]));
  }
}

template <typename T, int NF, int TY, int NST>
__global__ void __launch_bounds__(32 * (TY + 1), (min_blocks<T, NF, TY, NST>()))
    k_step_sweep(const StepArgs<T> p, const __grid_constant__ SweepMaps maps) {
  constexpr int VX = 16 / sizeof(T);     // sites per thread (one 16-byte vector)
  constexpr int TX = 32 * VX;            // tile width: one warp per row
  constexpr int H = VX;                  // x-halo box width (16 bytes)
  constexpr int MAIN = (TY + 2) * TX;    // tile + y-halo rows, elements
  constexpr int HALO = (int)(halo_bytes(TY) / sizeof(T));  // one x-halo column buffer, elements
  constexpr int ARR = MAIN + 2 * HALO;   // + left and right x-halo columns
  constexpr uint32_t kPlaneBytes = 2u * NF * (MAIN + 2 * TY * H) * sizeof(T);  // bytes TMA delivers per plane
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  // TMA destinations are kept 128-byte aligned whatever the static smem layout.
  unsigned char* smem_raw = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~static_cast<uintptr_t>(127));
  T* stage = reinterpret_cast<T*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)NST * NF * 2 * ARR * sizeof(T));
  uint64_t* empty = full + NST;
  uint64_t* gready = empty + NST;   // all consumer warps wrote their g rows into a slot
  __shared__ int s_abort;
  __shared__ int s_min_waited;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const bool producer = (warp == TY);
  const int r = warp;  // consumer warp r owns tile row r
  const int N = (int)p.N;
  const int64_t NN = (int64_t)N * N;
  const int x0 = blockIdx.x * TX;
  const int y0 = blockIdx.y * TY;
  const int z0 = (int)(((int64_t)blockIdx.z * N) / gridDim.z);
  const int z1 = (int)(((int64_t)(blockIdx.z + 1) * N) / gridDim.z);
  const int nplanes = z1 - z0 + 2;  // planes z0-1 .. z1
  // Neighbouring z-chunks sweep in opposite directions, so the two chunks that
  // share a boundary plane read it at about the same time (the second read
  // hits L2).  Plane index k of the sweep is z0 - 1 + k upwards, z1 - k downwards.
  const bool down = (blockIdx.z & 1u) != 0;
  auto plane_z = [&](int k) { return down ? z1 - k : z0 - 1 + k; };

  auto sbuf = [&](int slot, int i, int a) -> T* {
    return stage + ((size_t)(slot * NF + i) * 2 + a) * ARR;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TY);
      mbar_init(&gready[s], TY);
    }
    s_abort = 0;
    s_min_waited = nplanes;
    fence_mbar_init();
  }
  __syncthreads();

  // Bounded wait: gives up when another warp aborted or after ~2 s of clock.
  auto wait_bar = [&](uint64_t* bar, uint32_t parity) -> bool {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
      if (*(volatile int*)&s_abort) return false;
      if (clock64() - t0 > p.wait_cycles) {
        atomicExch(&s_abort, 1);
        atomicCAS(p.status, CE_OK, CE_ETIMEOUT);
        return false;
      }
    }
    return true;
  };

  double grad2 = 0.0, pot = 0.0;
  int issued = 0;
  if (producer) {
    // ---------------- producer warp: one lane streams planes into the ring
    if (lane == 0) {
      const int xl = (x0 == 0) ? N - H : x0 - H;
      const int xr = (x0 + TX == N) ? 0 : x0 + TX;
      for (int pidx = 0; pidx < nplanes; ++pidx) {
        const int slot = pidx % NST;
        if (pidx >= NST && !wait_bar(&empty[slot], (uint32_t)(pidx / NST - 1) & 1u)) break;
        int zz = plane_z(pidx);
        zz = zz < 0 ? zz + N : (zz >= N ? zz - N : zz);
        mbar_expect_tx(&full[slot], kPlaneBytes + p.missing_tx);
#pragma unroll
        for (int i = 0; i < NF; ++i) {
#pragma unroll
          for (int a = 0; a < 2; ++a) {
            T* dst = sbuf(slot, i, a);
            if (y0 == 0) {
              tma_load_3d(dst + TX, &maps.m[i][a][1], x0, 0, zz, &full[slot]);
              tma_load_3d(dst, &maps.m[i][a][2], x0, N - 1, zz, &full[slot]);
            } else if (y0 + TY == N) {
              tma_load_3d(dst, &maps.m[i][a][1], x0, y0 - 1, zz, &full[slot]);
              tma_load_3d(dst + (TY + 1) * TX, &maps.m[i][a][2], x0, 0, zz, &full[slot]);
            } else {
              tma_load_3d(dst, &maps.m[i][a][0], x0, y0 - 1, zz, &full[slot]);
            }
            tma_load_3d(dst + MAIN, &maps.m[i][a][3], xl, y0, zz, &full[slot]);
            tma_load_3d(dst + MAIN + HALO, &maps.m[i][a][3], xr, y0, zz, &full[slot]);
          }
        }
        issued = pidx + 1;
      }
    }
  } else {
    // ---------------- consumer warps: one tile row each, sweeping z
    const T c = (T)p.sc_in->c;
    const T dd = p.dt_drift, kk = p.dt_kick, idx2 = p.inv_dx2;
    T q[3] = {p.q[0], p.q[1], p.q[2]};
    const int col = lane * VX;
    T g2loc = T(0), vloc = T(0);
    T gp[NF][VX], gc[NF][VX], vc[NF][VX];
    int waited = 0;
    // A slot goes back to the producer once nobody reads it; the consumers also
    // wrote g rows into it, which the next TMA fill overwrites.
    auto release = [&](int pidx) {
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[pidx % NST]);
    };
    // Each warp replaces the f of its own staged row by g = f + dt (w + c f)
    // (warps 0 and TY-1 also convert the y-halo rows), so the rows above and
    // below read their y-neighbours' g instead of recomputing it from f and w;
    // the g values are the same numbers either way.  gready[slot] completes
    // when all TY warps have written the slot (every plane position, written
    // or not, so its phases stay in step with the ring).
    auto put_g = [&](int slot, const T (&g)[NF][VX]) {
#pragma unroll
      for (int i = 0; i < NF; ++i) sts16<T, VX>(sbuf(slot, i, 0) + (r + 1) * TX + col, g[i]);
      if (r == 0 || r == TY - 1) {
        const int hr = (r == 0) ? 0 : TY + 1;
#pragma unroll
        for (int i = 0; i < NF; ++i) {
          T f[VX], w[VX], h[VX];
          lds16<T, VX>(sbuf(slot, i, 0) + hr * TX + col, f);
          lds16<T, VX>(sbuf(slot, i, 1) + hr * TX + col, w);
#pragma unroll
          for (int j = 0; j < VX; ++j) h[j] = fmaT(dd, fmaT(c, f[j], w[j]), f[j]);
          sts16<T, VX>(sbuf(slot, i, 0) + hr * TX + col, h);
        }
      }
    };
    auto publish = [&](int pidx) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&gready[pidx % NST]);
    };
    bool ok = __all_sync(0xffffffffu, wait_bar(&full[0], 0u));
    if (ok) {
      waited = 1;
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        T f[VX], w[VX];
        lds16<T, VX>(sbuf(0, i, 0) + (r + 1) * TX + col, f);
        lds16<T, VX>(sbuf(0, i, 1) + (r + 1) * TX + col, w);
#pragma unroll
        for (int j = 0; j < VX; ++j) gp[i][j] = fmaT(dd, fmaT(c, f[j], w[j]), f[j]);
      }
      publish(0);   // plane 0 is only a z-neighbour: no g rows needed
      release(0);
      ok = __all_sync(0xffffffffu, wait_bar(&full[1 % NST], (uint32_t)(1 / NST) & 1u));
    }
    if (ok) {
      waited = 2;
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        T f[VX], w[VX];
        lds16<T, VX>(sbuf(1 % NST, i, 0) + (r + 1) * TX + col, f);
        lds16<T, VX>(sbuf(1 % NST, i, 1) + (r + 1) * TX + col, w);
#pragma unroll
        for (int j = 0; j < VX; ++j) {
          vc[i][j] = fmaT(c, f[j], w[j]);
          gc[i][j] = fmaT(dd, vc[i][j], f[j]);
        }
      }
      put_g(1 % NST, gc);
      publish(1);
    }
    for (int pc = 1; pc <= nplanes - 2 && ok; ++pc) {
      const int z = plane_z(pc);  // the plane computed now
      const int pn = pc + 1;      // the next plane of the sweep (z +- 1)
      if (!__all_sync(0xffffffffu, wait_bar(&full[pn % NST], (uint32_t)(pn / NST) & 1u))) {
        ok = false;
        break;
      }
      waited = pn + 1;
      const int sc_cur = pc % NST, sc_nxt = pn % NST;
      // gp / gc / gn: g at the previous, current and next plane of the sweep
      T gn[NF][VX], vn[NF][VX], lap[NF][VX];
#pragma unroll
      for (int i = 0; i < NF; ++i) {  // next plane, own sites
        T f[VX], w[VX];
        lds16<T, VX>(sbuf(sc_nxt, i, 0) + (r + 1) * TX + col, f);
        lds16<T, VX>(sbuf(sc_nxt, i, 1) + (r + 1) * TX + col, w);
#pragma unroll
        for (int j = 0; j < VX; ++j) {
          vn[i][j] = fmaT(c, f[j], w[j]);
          gn[i][j] = fmaT(dd, vn[i][j], f[j]);
        }
      }
      if (pn <= nplanes - 2) put_g(sc_nxt, gn);   // the last plane is only a z-neighbour
      publish(pn);
      // the current plane's g rows, written by all warps one plane ago
      if (!__all_sync(0xffffffffu, wait_bar(&gready[sc_cur], (uint32_t)(pc / NST) & 1u))) {
        ok = false;
        break;
      }
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        const T* cf = sbuf(sc_cur, i, 0);
        const T* cw = sbuf(sc_cur, i, 1);
        T ym[VX], yp[VX];
        lds16<T, VX>(cf + r * TX + col, ym);          // g of the row below (y - 1)
        lds16<T, VX>(cf + (r + 2) * TX + col, yp);    // g of the row above (y + 1)
        // x neighbours: adjacent lanes; the row ends read the TMA'd halo columns
        const int hoff = (lane == 0) ? MAIN + r * H + (H - 1) : MAIN + HALO + r * H;
        const T hf = cf[hoff], hw = cw[hoff];
        const T gh = fmaT(dd, fmaT(c, hf, hw), hf);
        T gl = __shfl_up_sync(0xffffffffu, gc[i][VX - 1], 1);
        T gr = __shfl_down_sync(0xffffffffu, gc[i][0], 1);
        if (lane == 0) gl = gh;
        if (lane == 31) gr = gh;
#pragma unroll
        for (int j = 0; j < VX; ++j) {
          const T g = gc[i][j];
          const T xm = (j == 0) ? gl : gc[i][j - 1];
          const T xp = (j == VX - 1) ? gr : gc[i][j + 1];
          if constexpr (sizeof(T) == 8) {
            // FP64 (bound by the FP64 pipe): the six neighbours summed once, and
            // the gradient energy by summation by parts on the periodic lattice,
            //   sum_x sum_d (g(x+e_d) - g(x))^2 = -sum_x g(x) raw(x),
            //   raw(x) = sum_d (g(x+e_d) + g(x-e_d) - 2 g(x)),
            // one FMA per site instead of six operations.  The cancellation in
            // the sum costs about 1e-12 of G in FP64, which enters only a''.
            const T raw = fmaT(T(-6), g, ((xp + xm) + (yp[j] + ym[j])) + (gn[i][j] + gp[i][j]));
            lap[i][j] = raw * idx2;
            g2loc = fmaT(-g, raw, g2loc);
          } else {
            T acc = T(0);
            acc += (xp + xm) - T(2) * g;
            acc += (yp[j] + ym[j]) - T(2) * g;
            acc += (gn[i][j] + gp[i][j]) - T(2) * g;
            lap[i][j] = acc * idx2;
            const T dx = xp - g, dy = yp[j] - g, dz = (down ? gp[i][j] : gn[i][j]) - g;
            g2loc = fmaT(dx, dx, g2loc);
            g2loc = fmaT(dy, dy, g2loc);
            g2loc = fmaT(dz, dz, g2loc);
          }
        }
      }
      release(pc);  // plane z is no longer read
      const int64_t out = (int64_t)z * NN + (int64_t)(y0 + r) * N + x0 + col;
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        T gs[NF], dv[NF], vs;
#pragma unroll
        for (int i = 0; i < NF; ++i) gs[i] = gc[i][j];
        model_dv<T, NF>(gs, q, dv, vs);
        vloc += vs;
#pragma unroll
        for (int i = 0; i < NF; ++i) lap[i][j] = fmaT(kk, lap[i][j] - dv[i], vc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        stg16<T, VX>(p.f_out[i] + out, gc[i]);
        stg16<T, VX>(p.w_out[i] + out, lap[i]);
      }
#pragma unroll
      for (int i = 0; i < NF; ++i) {
#pragma unroll
        for (int j = 0; j < VX; ++j) {
          gp[i][j] = gc[i][j];
          gc[i][j] = gn[i][j];
          vc[i][j] = vn[i][j];
        }
      }
    }
    if (lane == 0) atomicMin(&s_min_waited, waited);
    grad2 = (double)g2loc;
    pot = (double)vloc;
  }
  __syncthreads();
  if (s_abort) {
    // Give the copies still in flight a bounded chance to land before the CTA's
    // shared memory is released; the sums of this launch are void.
    if (threadIdx.x == TY * 32) {
      for (int k = s_min_waited; k < issued; ++k) {
        const long long t0 = clock64();
        while (!mbar_try_wait(&full[k % NST], (uint32_t)(k / NST) & 1u) && clock64() - t0 < p.wait_cycles) {
        }
      }
    }
    __syncthreads();
    grad2 = 0.0;
    pot = 0.0;
  }
  if (p.update_scalars) finish_step_block(p, grad2, pot);
}


}  // namespace sweep
}  // namespace ce
