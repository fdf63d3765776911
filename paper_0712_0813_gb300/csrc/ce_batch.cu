// ce_batch.cu -- one leapfrog step of many lattices (any mix of 1D/2D/3D and
// sizes) in a single persistent launch, and the ce_batch_* C ABI around it.
//
// Per site the arithmetic is the fused step of the single-lattice kernels
// (arXiv:0712.0813 Sec. III staggered leapfrog): v = w + c f, g = f + dt v,
// w_out = v + dt (lap g - dV/df(g)), f_out = g, plus the sums of
// (g(x+e_d) - g(x))^2 and V(g) that advance each lattice's own scale factor.
//
// Work decomposition.  Every 2D and 3D lattice of the batch is cut into work
// items of about the same size, and a CTA of 8 warps takes one item, swept
// along the lattice's slowest axis (z in 3D, y in 2D).  3D: rows of one segment
// of 32, 16 or 8 lanes x VX sites (VX = 16 B / sizeof(T); the width that pads a
// row of N sites least), so a warp holds 1, 2 or 4 rows; 2D: each warp owns one
// 32-lane segment of a row.  Each plane of the item (f and w of every field, in
// 3D with the two y-halo rows and the x-halo columns) is staged in a
// shared-memory ring: 3D planes by TMA tensor copies from per-lattice tensor
// maps (one lane per field and array issues the boxes, an mbarrier per slot
// signals their arrival), 2D planes by per-thread cp.async.  One block barrier per plane publishes the landed plane and frees
// the slot read two planes earlier.  Sweep-axis neighbours stay in registers,
// x-neighbours come from the adjacent lane by shuffle and from the staged halo,
// y-neighbours from the staged rows.  Segments may be partial (N not a multiple
// of the segment): lanes past the row end idle.
//
// The grid is persistent: a fixed number of resident CTAs pull items from one
// queue (an atomic counter), largest items first.  The CTA that completes the
// last item of a lattice combines that lattice's item partials (all its
// threads, in an order fixed by the lattice's item count) and advances its a,
// a', a'' -- nobody waits for anybody.  The last CTA to
// leave resets the queue for the next launch.
//
// 1D lattices have no plane to sweep and little work per row segment: staged
// one segment span at a time they streamed HBM at a quarter of the bandwidth.
// They run in a second kernel, k_step_1d_members (the single-lattice 1D
// kernel's per-group arithmetic, 16-byte loads and stores straight from HBM,
// each block kG1d x 256 groups of VX sites of one lattice); each lattice's last
// block combines its blocks' sums and advances its scale factor.  The 1D and
// the 2D/3D lattices share nothing, so the 1D launches go on a second stream
// forked from the batch's stream (and joined back after the step loop, also
// inside the captured graphs): they run while the persistent kernel leaves SMs
// free, at its tail.  Step loops are CUDA graphs of 32 steps.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <string>
#include <vector>

#include "ce_device.cuh"
#include "ce_internal.h"
#include "ce_plan.h"
#include "ce_tma.cuh"

namespace ce {
namespace {

constexpr int kWarps = plan::kRowWarps;   // 8 (the launch models in ce_plan.h assume it)
constexpr int kThreads = 32 * kWarps;
// Tensor-map box shapes of a 3D member, per (buffer parity, field, f or w):
// row boxes one segment wide and rows + 2, rows + 1, 1, nlast + 1 and nlast
// rows high (nlast: rows of the lattice's last row group), then x-halo column
// boxes 16 bytes wide and rows or nlast rows high.
constexpr int kMapTypes = 7;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz: bound of every device-side wait
constexpr int kBatchGraphSteps = 32;
constexpr int kG1d = 4;   // groups of VX sites per thread of the 1D launch

template <typename T>
struct BMember {
  T* f[2][4];
  T* w[2][4];
  DevScalars* slot;        // the lattice's two scalar slots
  int* status;
  unsigned int* done;      // items of this lattice completed in the running launch
  double* partials;        // 2 doubles per item of this lattice
  int dims, N, p0, first_item, n_items, update_scalars;   // 1D: n_items = blocks of the 1D launch
  int seg_log2;            // 3D: log2 of the lanes per row segment (5, 4 or 3: 1, 2 or 4 rows per warp)
  const CUtensorMap* tmaps;  // 3D: tensor maps of f, w (see kMapTypes), device memory; else null
  T inv_dx2, dt, q[3];
  double ddt, kappa2, inv_S, half_inv_dx2;
};

struct BItem {
  int member;
  int x0;      // first x site of the (first) segment
  int y0;      // first row (3D items)
  int s0, s1;  // sweep range: z (3D), y (2D)
};

template <typename T, int VX>
__device__ __forceinline__ void st16(T* p, const T (&o)[VX]) {
  if constexpr (sizeof(T) == 4) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(o[0], o[1], o[2], o[3]));
  } else {
    __stcs(reinterpret_cast<double2*>(p), make_double2(o[0], o[1]));
  }
}

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

// Shared-memory layout of one array (f or w of one field) in one ring stage.
// 3D: the item's rows plus the two y-halo rows, each one segment wide (a
// segment is LR = 32, 16 or 8 lanes x VX sites, so a warp holds 1, 2 or 4 rows
// and an item rows = 8, 16 or 32 rows: (rows + 2) W sites, which is 8 SEG + 2 W),
// then the left and the right x-halo columns, 16 bytes (VX sites) per row each,
// as TMA delivers them.  2D: row 0 holds the 8 warps' segments side by side
// and the span's two halo elements follow the 10th row.  The largest 3D case
// (10 rows of 32 VX plus 2 x 8 x VX halo sites, or 34 rows of 8 VX plus
// 2 x 32 x VX) sizes the stage; ARR x sizeof(T) is a multiple of 128 bytes, so
// every TMA destination stays 128-byte aligned.
template <typename T>
struct Stage {
  static constexpr int VX = 16 / sizeof(T);
  static constexpr int SEG = 32 * VX;
  static constexpr int ARR = 10 * SEG + 16 * VX;
  static_assert((ARR * sizeof(T)) % 128 == 0, "stage arrays must keep TMA destinations 128-byte aligned");
};

template <typename T, int NF, int NST>
constexpr size_t batch_smem() {
  return (size_t)NST * NF * 2 * Stage<T>::ARR * sizeof(T) + 128;   // + alignment slack
}

// One item, processed by the whole CTA: a ring of NST stages keeps up to
// NST - 2 planes in flight while one is computed; one block barrier per plane
// both publishes the landed plane and frees the slot read two planes earlier.
// 3D planes arrive by TMA (one lane per array issues one or two row boxes and two
// x-halo column boxes from the member's tensor maps; full[slot] completes
// when the bytes have landed, every thread waits on it with a bounded wait and
// keeps the slot's phase in bit slot of ph); 2D planes by per-thread
// cp.async.  Returns false when a wait ran out (the caller stops).
// DIMS 3: a row segment is LR = 2^seg_log2 lanes x VX sites; lane l of warp w
// owns row r = w (32 / LR) + l / LR of the item, sites (l mod LR) VX .. + VX - 1
// of the segment, and sweeps z (x-neighbour shuffles stay inside each LR-lane
// group); DIMS 2: warp w owns segment w of an 8-segment span of one row and
// sweeps y.
template <typename T, int NF, int NST, int DIMS>
__device__ __forceinline__ bool run_item(const BMember<T>* __restrict__ m, int in, const BItem& it, T* smem,
                                         uint64_t* full, uint32_t& ph, int warp, int lane, T& g2loc, T& vloc) {
  static_assert(DIMS == 2 || DIMS == 3, "1D lattices run in k_step_1d_members");
  constexpr int VX = Stage<T>::VX, SEG = Stage<T>::SEG, ARR = Stage<T>::ARR;
  const int N = m->N;
  const int64_t NN = (int64_t)N * N;
  // geometry of this warp
  int x0, nvl, nrows = 8;
  // 3D segment geometry: lr lanes per row segment (32, 16 or 8), W sites wide
  int lr = 32, sub = lane, r = warp, W = SEG, hbase = 10 * SEG;
  bool wvalid, rvalid;
  if constexpr (DIMS == 3) {
    const int sl = m->seg_log2;
    lr = 1 << sl;
    sub = lane & (lr - 1);
    r = (warp << (5 - sl)) + (lane >> sl);
    W = lr * VX;
    const int rows = 8 << (5 - sl);
    hbase = (rows + 2) * W;
    nrows = min(rows, N - it.y0);
    wvalid = (warp << (5 - sl)) < nrows;
    rvalid = r < nrows;
    x0 = it.x0;
    nvl = min(lr, (N - x0) / VX);
  } else {
    x0 = it.x0 + warp * SEG;
    wvalid = x0 < N;
    rvalid = wvalid;
    nvl = wvalid ? min(32, (N - x0) / VX) : 0;
  }
  const bool valid = rvalid && sub < nvl;
  const int col = sub * VX;                      // column inside the lane's segment
  const int span_end = min(N, it.x0 + 8 * SEG);  // 2D: end of the CTA's span
  const int last_warp = (span_end - it.x0 + SEG - 1) / SEG - 1;
  const int y = it.y0 + r;                       // 3D row
  const auto wrap = [&](int v) { return v < 0 ? v + N : (v >= N ? v - N : v); };
  const int n = it.s1 - it.s0 + 2;
  const auto plane = [&](int j) { return wrap(it.s0 - 1 + j); };
  const T c = (T)m->slot[in].c;
  const T dd = m->dt, kk = m->dt, idx2 = m->inv_dx2;
  T q[3] = {m->q[0], m->q[1], m->q[2]};
  const auto sbuf = [&](int slot, int i, int a) { return smem + ((size_t)(slot * NF + i) * 2 + a) * ARR; };

  const int own_row = DIMS == 3 ? (r + 1) * W + col : warp * SEG + col;
  // 3D: the staged rows 0 .. nrows + 1 hold lattice rows y0 - 1 .. y0 + nrows
  // (mod N): one box where they do not wrap, else a box per contiguous run;
  // box heights are those of the member's tensor maps (kMapTypes).  The x-halo
  // columns are the 16-byte chunks holding sites x0 - 1 and x0 + len (mod N).
  const int rows3 = DIMS == 3 ? 8 << (5 - m->seg_log2) : 8;
  const uint32_t plane_bytes =
      (uint32_t)(NF * 2 * ((nrows + 2) * W * (int)sizeof(T) + 2 * nrows * 16));
  const auto issue = [&](int j) {
    const int slot = j % NST;
    if constexpr (DIMS == 3) {
      // thread 0 posts the plane's bytes; lane 0 of warp w issues the boxes of
      // field w / 2, array (f, w) w % 2 (a complete_tx may run ahead of the
      // expect_tx: the phase cannot end before thread 0's arrival)
      if (threadIdx.x == 0) mbar_expect_tx(&full[slot], plane_bytes);
      if (lane != 0 || warp >= 2 * NF) return;
      const int i = warp >> 1, a = warp & 1;
      const int zz = plane(j);
      const int y0 = it.y0;
      const int len = min(W, N - x0);
      const int xl = x0 >= VX ? x0 - VX : N - VX, xr = x0 + len < N ? x0 + len : 0;
      const int hts = nrows == rows3 ? 5 : 6;        // x-halo map: rows or nlast rows high
      T* st = sbuf(slot, i, a);
      const CUtensorMap* mp = m->tmaps + ((in * NF + i) * 2 + a) * kMapTypes;
      if (y0 >= 1 && y0 + nrows <= N - 1) {          // no wrap: rows y0-1 .. y0+rows
        tma_load_3d(st, mp + 0, x0, y0 - 1, zz, &full[slot]);
      } else if (y0 == 0 && nrows < N) {            // first group: row N-1, then 0 .. rows
        tma_load_3d(st, mp + 2, x0, N - 1, zz, &full[slot]);
        tma_load_3d(st + W, mp + 1, x0, 0, zz, &full[slot]);
      } else if (y0 == 0) {                         // one group holds every row
        tma_load_3d(st, mp + 2, x0, N - 1, zz, &full[slot]);
        tma_load_3d(st + W, mp + 4, x0, 0, zz, &full[slot]);
        tma_load_3d(st + (nrows + 1) * W, mp + 2, x0, 0, zz, &full[slot]);
      } else {                                      // last group: rows y0-1 .. N-1, then row 0
        tma_load_3d(st, mp + 3, x0, y0 - 1, zz, &full[slot]);
        tma_load_3d(st + (nrows + 1) * W, mp + 2, x0, 0, zz, &full[slot]);
      }
      tma_load_3d(st + hbase, mp + hts, xl, y0, zz, &full[slot]);
      tma_load_3d(st + hbase + rows3 * VX, mp + hts, xr, y0, zz, &full[slot]);
      return;
    } else {
      const int64_t poff = (int64_t)plane(j) * N;
#pragma unroll
      for (int i = 0; i < NF; ++i) {
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const T* base = (a ? m->w[in][i] : m->f[in][i]) + poff;
          T* st = sbuf(slot, i, a);
          {
            if (valid) cp16(st + warp * SEG + col, base + x0 + col);
            if (warp == 0 && lane == 0) cp_small<sizeof(T)>(st + 10 * SEG, base + wrap(it.x0 - 1));
            if (warp == last_warp && lane == nvl - 1)
              cp_small<sizeof(T)>(st + 10 * SEG + 1, base + (span_end == N ? 0 : span_end));
          }
        }
      }
    }
  };
  // 3D: bounded wait for plane j's bytes (~2 s of clock); keeps the slot phase.
  const auto wait_plane = [&](int j) -> bool {
    const int slot = j % NST;
    const uint32_t parity = (ph >> slot) & 1u;
    const long long t0 = clock64();
    while (!mbar_try_wait(&full[slot], parity))
      if (clock64() - t0 > kWaitCycles) return false;
    ph ^= 1u << slot;
    return true;
  };
  const auto gval = [&](T f, T w) { return fmaT(dd, fmaT(c, f, w), f); };

  // one plane's update at the own sites from registers (gp, gc, gn) and the
  // staged current plane (y and x neighbours, and the own sites' f, w again for
  // v = w + c f: recomputing it is cheaper than holding it in registers)
  T gp[NF][VX], gc[NF][VX];
  const auto update = [&](int j, const T (&gn)[NF][VX]) {
    const int slot = j % NST;
    const int zj = plane(j);
    T lap[NF][VX];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      const T* cf = sbuf(slot, i, 0);
      const T* cw = sbuf(slot, i, 1);
      T ym[VX], yp[VX];
      if constexpr (DIMS == 3) {
        T f[VX], w[VX];
        lds16<T, VX>(cf + r * W + col, f);
        lds16<T, VX>(cw + r * W + col, w);
#pragma unroll
        for (int k = 0; k < VX; ++k) ym[k] = gval(f[k], w[k]);
        lds16<T, VX>(cf + (r + 2) * W + col, f);
        lds16<T, VX>(cw + (r + 2) * W + col, w);
#pragma unroll
        for (int k = 0; k < VX; ++k) yp[k] = gval(f[k], w[k]);
      }
      // x neighbours: adjacent lanes; segment ends from the staged row or the halo
      T hl, hr;
      if constexpr (DIMS == 3) {
        const int li = hbase + r * VX + (VX - 1), ri = hbase + rows3 * VX + r * VX;
        hl = gval(cf[li], cw[li]);
        hr = gval(cf[ri], cw[ri]);
      } else {
        const int li = warp > 0 ? warp * SEG - 1 : 10 * SEG;
        const bool inner_r = x0 + nvl * VX < span_end;
        const int ri = inner_r ? warp * SEG + nvl * VX : 10 * SEG + 1;
        hl = gval(cf[li], cw[li]);
        hr = gval(cf[ri], cw[ri]);
      }
      T gl = __shfl_up_sync(0xffffffffu, gc[i][VX - 1], 1, lr);
      T gr = __shfl_down_sync(0xffffffffu, gc[i][0], 1, lr);
      if (sub == 0) gl = hl;
      if (sub == nvl - 1) gr = hr;
#pragma unroll
      for (int k = 0; k < VX; ++k) {
        const T g = gc[i][k];
        const T xm = (k == 0) ? gl : gc[i][k - 1];
        const T xp = (k == VX - 1) ? gr : gc[i][k + 1];
        T acc = T(0);
        acc += (xp + xm) - T(2) * g;
        T d2 = (xp - g) * (xp - g);
        if constexpr (DIMS == 3) {
          acc += (yp[k] + ym[k]) - T(2) * g;
          acc += (gn[i][k] + gp[i][k]) - T(2) * g;
          d2 = fmaT(yp[k] - g, yp[k] - g, d2);
          d2 = fmaT(gn[i][k] - g, gn[i][k] - g, d2);
        } else if constexpr (DIMS == 2) {
          acc += (gn[i][k] + gp[i][k]) - T(2) * g;
          d2 = fmaT(gn[i][k] - g, gn[i][k] - g, d2);
        }
        lap[i][k] = acc * idx2;
        if (valid) g2loc += d2;
      }
    }
    T vc[NF][VX];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      T f[VX], w[VX];
      if (valid) {
        lds16<T, VX>(sbuf(slot, i, 0) + own_row, f);
        lds16<T, VX>(sbuf(slot, i, 1) + own_row, w);
      } else {
#pragma unroll
        for (int k = 0; k < VX; ++k) f[k] = w[k] = T(0);
      }
#pragma unroll
      for (int k = 0; k < VX; ++k) vc[i][k] = fmaT(c, f[k], w[k]);
    }
#pragma unroll
    for (int k = 0; k < VX; ++k) {
      T gs[NF], dv[NF], vs;
#pragma unroll
      for (int i = 0; i < NF; ++i) gs[i] = gc[i][k];
      model_dv<T, NF>(gs, q, dv, vs);
      if (valid) vloc += vs;
#pragma unroll
      for (int i = 0; i < NF; ++i) lap[i][k] = fmaT(kk, lap[i][k] - dv[i], vc[i][k]);
    }
    if (valid) {
      const int64_t here = DIMS == 3 ? (int64_t)zj * NN + (y * N + x0 + col) : (int64_t)zj * N + x0 + col;
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        st16<T, VX>(m->f[in ^ 1][i] + here, gc[i]);
        st16<T, VX>(m->w[in ^ 1][i] + here, lap[i]);
      }
    }
  };
  const auto own_g = [&](int j, T (&g)[NF][VX]) {
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      T f[VX], w[VX];
      if (valid) {
        lds16<T, VX>(sbuf(j % NST, i, 0) + own_row, f);
        lds16<T, VX>(sbuf(j % NST, i, 1) + own_row, w);
      } else {
#pragma unroll
        for (int k = 0; k < VX; ++k) f[k] = w[k] = T(0);
      }
#pragma unroll
      for (int k = 0; k < VX; ++k) g[i][k] = fmaT(dd, fmaT(c, f[k], w[k]), f[k]);
    }
  };

  // prologue: fill the ring (3D: every thread's fence, then the barrier, order
  // a previous 2D item's cp.async writes into the same slots before these
  // TMA writes)
  if constexpr (DIMS == 3) {
    fence_proxy_async_smem();
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < NST; ++j) {
    if (j < n) issue(j);
    if constexpr (DIMS != 3) cp_commit();
  }
  int issued = min(n, NST), waited = 0;
  // 3D: every thread waits for plane j's bytes, then the block barrier; when a
  // wait ran out, all threads stop and thread 0 waits (bounded) for the copies
  // still in flight, so no TMA write lands after the CTA's shared memory is gone.
  const auto landed = [&](int j) -> bool {
    const bool ok = wait_plane(j);
    if (ok) waited = j + 1;
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0)
        for (int pl = waited; pl < issued; ++pl) wait_plane(pl);
      return false;
    }
    return true;
  };
  {
    if constexpr (DIMS == 3) {
      if (!landed(0) || !landed(1)) return false;
    } else {
      cp_wait<NST - 2>();   // planes 0 and 1 have landed
      __syncthreads();
    }
    if (wvalid) {
      own_g(0, gp);
      own_g(1, gc);
    }
    for (int j = 1; j <= n - 2; ++j) {
      if constexpr (DIMS == 3) {
        if (!landed(j + 1)) return false;   // plane j + 1 is in, plane j - 1's slot is free
      } else {
        cp_wait<NST - 3>();  // plane j + 1 has landed (own copies) ...
        __syncthreads();     // ... for every thread, and plane j - 1's slot is free
      }
      if (j + NST - 1 < n) {
        issue(j + NST - 1);
        issued = j + NST;
      }
      if constexpr (DIMS != 3) cp_commit();
      if (wvalid) {
        T gn[NF][VX];
        own_g(j + 1, gn);
        update(j, gn);
#pragma unroll
        for (int i = 0; i < NF; ++i)
#pragma unroll
          for (int k = 0; k < VX; ++k) {
            gp[i][k] = gc[i][k];
            gc[i][k] = gn[i][k];
          }
      }
    }
  }
  return true;
}

template <typename T, int NF, int NST>
__global__ void __launch_bounds__(kThreads, NF <= 2 ? 2 : 1) k_step_batched(const BMember<T>* __restrict__ members,
                                                            const BItem* __restrict__ items, int n_items,
                                                            unsigned int* queue, int par) {
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  // 128-byte aligned for the TMA destinations (an offset of the shared array,
  // so the pointer stays in the shared space)
  T* smem = reinterpret_cast<T*>(smem_dyn + ((128u - (smem_addr(smem_dyn) & 127u)) & 127u));
  __shared__ int s_item, s_last;
  __shared__ __align__(8) uint64_t s_full[NST];   // TMA completion of each ring slot (3D items)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int k = 0; k < NST; ++k) mbar_init(&s_full[k], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t ph = 0;   // phase bit of each s_full slot; the same in every thread
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&queue[0], 1u);
    __syncthreads();
    const int itx = s_item;
    if (itx >= n_items) break;
    const BItem it = items[itx];
    const BMember<T>* m = members + it.member;
    const int in = m->p0 ^ par;
    T g2loc = T(0), vloc = T(0);
    bool ok;
    if (m->dims == 3) ok = run_item<T, NF, NST, 3>(m, in, it, smem, s_full, ph, warp, lane, g2loc, vloc);
    else ok = run_item<T, NF, NST, 2>(m, in, it, smem, s_full, ph, warp, lane, g2loc, vloc);
    if (!ok) {   // a bounded wait ran out: report it on the lattice and stop this CTA
      if (threadIdx.x == 0) atomicCAS(m->status, CE_OK, CE_ETIMEOUT);
      break;
    }
    if (m->update_scalars) {
      double g2, pot;
      block_sum2_t<T>(g2loc, vloc, g2, pot);
      if (threadIdx.x == 0) {
        const int k = itx - m->first_item;
        m->partials[2 * k] = g2;
        m->partials[2 * k + 1] = pot;
        __threadfence();
        s_last = atomicAdd(m->done, 1u) == (unsigned int)(m->n_items - 1);
      }
      __syncthreads();
      if (s_last) {
        // last item of this lattice: the whole CTA combines the item partials
        // (thread t takes items t, t + blockDim, ..., then a fixed tree, so the
        // order depends on the lattice's item count alone) and advances a
        __threadfence();
        double G = 0.0, V = 0.0;
        for (int j = threadIdx.x; j < m->n_items; j += blockDim.x) {
          G += __ldcg(m->partials + 2 * j);
          V += __ldcg(m->partials + 2 * j + 1);
        }
        block_sum2(G, V);
        if (threadIdx.x == 0) {
          DevScalars out;
          scale_factor_update(m->slot[in], out, G * m->half_inv_dx2 * m->inv_S, V * m->inv_S, m->ddt,
                              m->kappa2, m->status);
          m->slot[in ^ 1] = out;
          *m->done = 0u;
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&queue[1], 1u) == gridDim.x - 1) {
      queue[0] = 0u;
      queue[1] = 0u;
      __threadfence();
    }
  }
}

// One step of the batch's 1D lattices: blockIdx.y picks the lattice (m1d
// lists the 1D members), blockIdx.x a block of kG1d x kThreads groups of VX
// sites inside it (thread t takes groups t, t + kThreads, ...; blocks past the
// lattice's n_items leave at once).  Per site the arithmetic is
// step1d_group's (that of the single-lattice 1D kernel); a thread's sums stay
// in T over its kG1d groups (16 sites in FP32, as in the other step kernels),
// the block adds them with block_sum2_t into the lattice's partials, and the
// lattice's last block adds those in block order (thread t takes blocks t, t +
// kThreads, ..., then a fixed tree) and advances its a, a', a''.  A lattice's
// blocks and the order of its sums depend on its N alone, so its result does
// not depend on the mix.
template <typename T, int NF>
__global__ void __launch_bounds__(kThreads) k_step_1d_members(const BMember<T>* __restrict__ members,
                                                              const int* __restrict__ m1d, int par) {
  constexpr int VX = 16 / sizeof(T);
  const BMember<T>* m = members + m1d[blockIdx.y];
  const int nb = m->n_items;
  if ((int)blockIdx.x >= nb) return;
  const int in = m->p0 ^ par;
  const int64_t N = m->N, groups = N / VX;
  const T q[3] = {m->q[0], m->q[1], m->q[2]};
  const T c = (T)m->slot[in].c;
  const T* f_in[4];
  const T* w_in[4];
  T* f_out[4];
  T* w_out[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f_in[i] = m->f[in][i];
    w_in[i] = m->w[in][i];
    f_out[i] = m->f[in ^ 1][i];
    w_out[i] = m->w[in ^ 1][i];
  }
  T g2loc = T(0), vloc = T(0);
  const int64_t k0 = (int64_t)blockIdx.x * (kG1d * kThreads) + threadIdx.x;
#pragma unroll
  for (int r = 0; r < kG1d; ++r) {
    const int64_t k = k0 + (int64_t)r * kThreads;
    if (k < groups)
      step1d_group<T, NF>(f_in, w_in, f_out, w_out, N, k, c, m->dt, m->dt, m->inv_dx2, q, g2loc, vloc);
  }
  if (!m->update_scalars) return;   // the same for every thread of the block
  __shared__ int s_last;
  double g2, pot;
  block_sum2_t<T>(g2loc, vloc, g2, pot);
  if (threadIdx.x == 0) {
    m->partials[2 * blockIdx.x] = g2;
    m->partials[2 * blockIdx.x + 1] = pot;
    __threadfence();
    s_last = atomicAdd(m->done, 1u) == (unsigned int)(nb - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double G = 0.0, V = 0.0;
  for (int j = threadIdx.x; j < nb; j += kThreads) {
    G += __ldcg(m->partials + 2 * j);
    V += __ldcg(m->partials + 2 * j + 1);
  }
  block_sum2(G, V);
  if (threadIdx.x == 0) {
    DevScalars out;
    scale_factor_update(m->slot[in], out, G * m->half_inv_dx2 * m->inv_S, V * m->inv_S, m->ddt, m->kappa2,
                        m->status);
    m->slot[in ^ 1] = out;
    *m->done = 0u;
  }
}

}  // namespace
}  // namespace ce

struct ce_batch {
  std::vector<ce_sim*> members;
  int prec = CE_F64, nf = 0, device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* d_members = nullptr;
  void* d_items = nullptr;
  unsigned int* d_queue = nullptr;   // [0] head, [1] exit count
  unsigned int* d_done = nullptr;    // per member
  double* d_partials = nullptr;      // 2 per item (and per block of a 1D member)
  int* d_m1d = nullptr;              // indices of the 1D members
  int n1d = 0, bx1d = 0;             // 1D members; blocks of the largest one
  int n_units = 0;                   // items plus the 1D members' blocks
  cudaStream_t side = nullptr;       // the 1D launches when the batch also has 2D/3D lattices
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void* d_maps = nullptr;            // tensor maps of the 3D members
  int n_items = 0, blocks = 0, par = 0, sweep_len = 32;
  int ctas_per_sm = 0;               // cap on resident CTAs per SM (0: as many as fit)
  int64_t sites = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graphs_ok = true;
  bool broken = false;   // a member was freed while in the batch
};

namespace {

int bfail(int code, const std::string& msg) {
  ce::set_last_error(msg);
  return code;
}

int bcuda(cudaError_t e, const char* what) {
  ce::set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return CE_ECUDA;
}

constexpr int kBatchStages = 4;

// One step: the persistent launch (2D/3D members) on the batch's stream and
// the 1D launch on `st1d` (the side stream, or the batch's stream itself).
template <typename T, int NF>
cudaError_t launch_nf(const ce_batch* b, int par, cudaStream_t st1d) {
  const auto* mem = static_cast<const ce::BMember<T>*>(b->d_members);
  const auto* it = static_cast<const ce::BItem*>(b->d_items);
  constexpr size_t smem = ce::batch_smem<T, NF, kBatchStages>();
  if (b->n_items > 0)
    ce::k_step_batched<T, NF, kBatchStages><<<b->blocks, ce::kThreads, smem, b->stream>>>(mem, it, b->n_items,
                                                                                           b->d_queue, par);
  if (b->n1d > 0)
    ce::k_step_1d_members<T, NF><<<dim3(b->bx1d, b->n1d), ce::kThreads, 0, st1d>>>(mem, b->d_m1d, par);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_t(const ce_batch* b, int par, cudaStream_t st1d) {
  switch (b->nf) {
    case 1: return launch_nf<T, 1>(b, par, st1d);
    case 2: return launch_nf<T, 2>(b, par, st1d);
    case 3: return launch_nf<T, 3>(b, par, st1d);
    default: return launch_nf<T, 4>(b, par, st1d);
  }
}

cudaError_t launch_batch(const ce_batch* b, int par) {
  cudaStream_t st1d = b->side ? b->side : b->stream;
  return b->prec == CE_F32 ? launch_t<float>(b, par, st1d) : launch_t<double>(b, par, st1d);
}

// Fork the side stream from the batch's stream / join it back (no-ops for a
// batch without a side stream).  Under stream capture these become the
// graph's fork and join edges.
cudaError_t fork_side(const ce_batch* b) {
  if (!b->side) return cudaSuccess;
  cudaError_t e = cudaEventRecord(b->ev_fork, b->stream);
  return e == cudaSuccess ? cudaStreamWaitEvent(b->side, b->ev_fork, 0) : e;
}
cudaError_t join_side(const ce_batch* b) {
  if (!b->side) return cudaSuccess;
  cudaError_t e = cudaEventRecord(b->ev_join, b->side);
  return e == cudaSuccess ? cudaStreamWaitEvent(b->stream, b->ev_join, 0) : e;
}

template <typename T, int NF>
cudaError_t prepare_nf(int* per_sm) {
  const void* k = (const void*)&ce::k_step_batched<T, NF, kBatchStages>;
  constexpr size_t smem = ce::batch_smem<T, NF, kBatchStages>();
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, ce::kThreads, smem);
  return e;
}

template <typename T>
cudaError_t prepare_t(int nf, int* per_sm) {
  switch (nf) {
    case 1: return prepare_nf<T, 1>(per_sm);
    case 2: return prepare_nf<T, 2>(per_sm);
    case 3: return prepare_nf<T, 3>(per_sm);
    default: return prepare_nf<T, 4>(per_sm);
  }
}

// Raise the kernel's shared-memory limit and report how many CTAs fit an SM.
cudaError_t batch_prepare(int prec, int nf, int* per_sm) {
  return prec == CE_F32 ? prepare_t<float>(nf, per_sm) : prepare_t<double>(nf, per_sm);
}


// Cut every 2D and 3D member into items of about kWarps x 32 x VX x sweep_len
// sites; a 1D member gets ceil(N / VX / kThreads) blocks of the 1D launch
// (listed in m1d).
template <typename T>
void build_tables(ce_batch* b, std::vector<ce::BMember<T>>& mem, std::vector<ce::BItem>& items,
                  std::vector<int>& m1d) {
  constexpr int VX = 16 / sizeof(T);
  constexpr int SEG = 32 * VX;
  struct Work {
    ce::BItem it;
    int64_t cost;
  };
  std::vector<std::vector<Work>> per(b->members.size());
  for (size_t k = 0; k < b->members.size(); ++k) {
    const ce_sim* s = b->members[k];
    const int N = (int)s->N;
    const int L = std::max(1, std::min(b->sweep_len, N));
    auto add = [&](int x0, int y0, int s0, int s1, int64_t cost) {
      per[k].push_back({ce::BItem{(int)k, x0, y0, s0, s1}, cost});
    };
    if (s->dims == 3) {
      const int sl = ce::plan::seg_log2_for(N, VX);
      const int W = VX << sl, rows = ce::kWarps << (5 - sl);
      // x-neighbouring items next to each other in the queue, then y: items that
      // share halo rows and halo sectors start together and read them from L2
      for (int z0 = 0; z0 < N; z0 += L)
        for (int y0 = 0; y0 < N; y0 += rows)
          for (int x0 = 0; x0 < N; x0 += W)
            add(x0, y0, z0, std::min(N, z0 + L), (int64_t)std::min(W, N - x0) * std::min(rows, N - y0) * (std::min(N, z0 + L) - z0));
    } else if (s->dims == 2) {
      for (int x0 = 0; x0 < N; x0 += ce::kWarps * SEG)
        for (int y0 = 0; y0 < N; y0 += L)
          add(x0, 0, y0, std::min(N, y0 + L), (int64_t)std::min(ce::kWarps * SEG, N - x0) * (std::min(N, y0 + L) - y0));
    }
  }
  // items of a member stay contiguous (their partials are indexed from first_item);
  // members are ordered by their largest item so the queue hands out big work first
  std::vector<size_t> order(b->members.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = k;
  const auto weight = [&](size_t k) { return per[k].empty() ? 0 : per[k].front().cost * (int64_t)per[k].size(); };
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) { return weight(a) > weight(c); });
  mem.resize(b->members.size());
  for (size_t k : order) {
    const ce_sim* s = b->members[k];
    ce::BMember<T>& m = mem[k];
    for (int p = 0; p < 2; ++p)
      for (int i = 0; i < 4; ++i) {
        const int ii = i < s->nf ? i : 0;
        m.f[p][i] = static_cast<T*>(s->f[p][ii]);
        m.w[p][i] = static_cast<T*>(s->w[p][ii]);
      }
    m.slot = s->aux->slot;
    m.status = &s->aux->status;
    m.done = b->d_done + k;
    m.dims = s->dims;
    m.N = (int)s->N;
    m.seg_log2 = s->dims == 3 ? ce::plan::seg_log2_for((int)s->N, VX) : 5;
    m.p0 = s->cur ^ b->par;
    m.first_item = (int)items.size();
    m.n_items = (int)per[k].size();
    if (s->dims == 1) {
      const int64_t per_block = (int64_t)ce::kG1d * ce::kThreads;
      m.n_items = (int)((s->N / VX + per_block - 1) / per_block);
      m1d.push_back((int)k);
    }
    m.update_scalars = s->cfg.expansion ? 1 : 0;
    m.inv_dx2 = (T)(1.0 / (s->dx * s->dx));
    m.dt = (T)s->cfg.dt;
    for (int i = 0; i < 3; ++i) m.q[i] = (T)s->cfg.q[i];
    m.ddt = s->cfg.dt;
    m.kappa2 = s->kappa2;
    m.inv_S = 1.0 / (double)s->S;
    m.half_inv_dx2 = 0.5 / (s->dx * s->dx);
    for (const Work& w : per[k]) items.push_back(w.it);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor maps of every 3D member's f and w (both buffer sets): the x/y/z box
// shapes of kMapTypes for the member's segment width and row-group height.
template <typename T>
int encode_maps(ce_batch* b, std::vector<ce::BMember<T>>& mem) {
  constexpr int VX = 16 / sizeof(T);
  size_t n3 = 0;
  for (const ce_sim* s : b->members) n3 += s->dims == 3;
  if (n3 == 0) return CE_OK;
  PFN_cuTensorMapEncodeTiled_v12000 enc = map_encoder();
  if (!enc) return bfail(CE_ECUDA, "ce_batch_create: no tensor-map encoder in the driver");
  const size_t per = (size_t)2 * b->nf * 2 * ce::kMapTypes;
  std::vector<CUtensorMap> maps(n3 * per);
  size_t at = 0;
  std::vector<size_t> first(b->members.size(), 0);
  for (size_t k = 0; k < b->members.size(); ++k) {
    const ce_sim* s = b->members[k];
    if (s->dims != 3) continue;
    first[k] = at;
    const int64_t N = s->N;
    const int sl = ce::plan::seg_log2_for((int)N, VX);
    const cuuint32_t W = (cuuint32_t)(VX << sl), rows = (cuuint32_t)(ce::kWarps << (5 - sl));
    const cuuint32_t groups = (cuuint32_t)((N + rows - 1) / rows);
    const cuuint32_t nlast = (cuuint32_t)(N - (int64_t)rows * (groups - 1));
    const cuuint32_t bw[ce::kMapTypes] = {W, W, W, W, W, (cuuint32_t)VX, (cuuint32_t)VX};
    const cuuint32_t bh[ce::kMapTypes] = {rows + 2, rows + 1, 1, nlast + 1, nlast, rows, nlast};
    const cuuint64_t gdim[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)N};
    const cuuint64_t gstride[2] = {(cuuint64_t)N * sizeof(T), (cuuint64_t)N * N * sizeof(T)};
    const cuuint32_t estride[3] = {1, 1, 1};
    for (int p = 0; p < 2; ++p)
      for (int i = 0; i < b->nf; ++i)
        for (int a = 0; a < 2; ++a)
          for (int t = 0; t < ce::kMapTypes; ++t) {
            const cuuint32_t box[3] = {bw[t], bh[t], 1};
            CUresult r = enc(&maps[at++], sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                             3, a == 0 ? s->f[p][i] : s->w[p][i], gdim, gstride, box, estride,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return bfail(CE_ECUDA, "ce_batch_create: tensor-map encoding failed");
          }
  }
  cudaError_t e = cudaMalloc(&b->d_maps, maps.size() * sizeof(CUtensorMap));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) return bcuda(e, "ce_batch_create: tensor maps");
  const CUtensorMap* dm = static_cast<const CUtensorMap*>(b->d_maps);
  for (size_t k = 0; k < b->members.size(); ++k)
    mem[k].tmaps = b->members[k]->dims == 3 ? dm + first[k] : nullptr;
  return CE_OK;
}

template <typename T>
int upload_tables(ce_batch* b) {
  std::vector<ce::BMember<T>> mem;
  std::vector<ce::BItem> items;
  std::vector<int> m1d;
  // partial-sum slots are assigned after the item count is known: the items'
  // first, then each 1D member's blocks
  build_tables<T>(b, mem, items, m1d);
  b->n_items = (int)items.size();
  b->n1d = (int)m1d.size();
  int64_t slots = b->n_items;
  for (int k : m1d) {
    mem[k].first_item = (int)slots;
    slots += mem[k].n_items;
    b->bx1d = std::max(b->bx1d, mem[k].n_items);
  }
  b->n_units = (int)slots;
  cudaError_t e = cudaMalloc(&b->d_partials, sizeof(double) * 2 * std::max<int64_t>(1, slots));
  if (e != cudaSuccess) return bcuda(e, "ce_batch_create: partials");
  for (auto& m : mem) m.partials = b->d_partials + 2 * (int64_t)m.first_item;
  if (b->n1d > 0) {
    e = cudaMalloc(&b->d_m1d, sizeof(int) * m1d.size());
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->d_m1d, m1d.data(), sizeof(int) * m1d.size(), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) return bcuda(e, "ce_batch_create: 1D member list");
  }
  if (int rc = encode_maps<T>(b, mem)) return rc;
  e = cudaMalloc(&b->d_members, sizeof(ce::BMember<T>) * mem.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(ce::BItem) * std::max<size_t>(1, items.size()));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_members, mem.data(), sizeof(ce::BMember<T>) * mem.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpyAsync(b->d_items, items.data(), sizeof(ce::BItem) * items.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e == cudaSuccess ? CE_OK : bcuda(e, "ce_batch_create: tables");
}

void release(ce_batch* b) {
  for (auto& g : b->graph)
    if (g) cudaGraphExecDestroy(g);
  if (b->d_members) cudaFree(b->d_members);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_queue) cudaFree(b->d_queue);
  if (b->d_partials) cudaFree(b->d_partials);
  if (b->d_maps) cudaFree(b->d_maps);
  if (b->d_m1d) cudaFree(b->d_m1d);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_join) cudaEventDestroy(b->ev_join);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

cudaError_t ensure_batch_graph(ce_batch* b, int start) {
  if (b->graph[start]) return cudaSuccess;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  cudaError_t el = fork_side(b);
  int par = start;
  for (int k = 0; k < ce::kBatchGraphSteps && el == cudaSuccess; ++k) {
    el = launch_batch(b, par);
    par ^= 1;
  }
  if (el == cudaSuccess) el = join_side(b);
  e = cudaStreamEndCapture(b->stream, &g);
  if (el != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return el != cudaSuccess ? el : e;
  }
  e = cudaGraphInstantiate(&b->graph[start], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) b->graph[start] = nullptr;
  return e;
}

void advance_members(ce_batch* b, int64_t steps) {
  for (ce_sim* s : b->members) {
    if (!s) continue;
    for (int64_t k = 0; k < steps; ++k) s->t = s->t + s->cfg.dt;
    s->step += steps;
    if (steps & 1) s->cur ^= 1;
  }
}

}  // namespace

cudaError_t ce::batch_wait(ce_batch* b) { return b ? cudaStreamSynchronize(b->stream) : cudaSuccess; }


// A private one-lattice batch that lets ce_step run the batched kernel on a
// single handle (lattices the z-sweep kernel does not cover).  It works on the
// handle's own stream, with step parity given per launch, and does not make
// the handle a batch member.
int ce::rows_create(ce_sim* s, ce_batch** out) {
  *out = nullptr;
  ce_batch* b = new (std::nothrow) ce_batch();
  if (!b) return bfail(CE_ENOMEM, "ce_create: host allocation");
  b->members.assign(1, s);
  b->prec = s->prec;
  b->nf = s->nf;
  b->device = s->device;
  b->sweep_len = 128;
  b->stream = s->stream;
  b->own_stream = false;
  b->par = 0;
  cudaError_t e = cudaMalloc(&b->d_queue, sizeof(unsigned int) * 3);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned int) * 3, b->stream);
  if (e != cudaSuccess) {
    release(b);
    delete b;
    return bcuda(e, "ce_create: row-kernel scratch");
  }
  b->d_done = b->d_queue + 2;
  // item length along the sweep axis: the candidate the launch model prefers
  int per_sm = 0, sms = 0;
  e = batch_prepare(b->prec, b->nf, &per_sm);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess || per_sm < 1) {
    release(b);
    delete b;
    return bcuda(e != cudaSuccess ? e : cudaErrorInvalidConfiguration, "ce_create: row-kernel occupancy");
  }
  b->sweep_len = ce::plan::rows_item_length(s->dims, s->N, 16 / s->esize, per_sm * sms);
  const int cur = s->cur;
  s->cur = 0;   // member parity 0: the launch's parity argument is the input buffer set
  int rc = b->prec == CE_F32 ? upload_tables<float>(b) : upload_tables<double>(b);
  s->cur = cur;
  if (rc != CE_OK) {
    release(b);
    delete b;
    return rc;
  }
  b->blocks = std::max(1, std::min(per_sm * sms, b->n_items));
  *out = b;
  return CE_OK;
}

cudaError_t ce::rows_launch(const ce_batch* b, int in, cudaStream_t st) {
  (void)st;   // the private batch was built on the handle's stream
  return launch_batch(b, in);
}

void ce::rows_free(ce_batch* b) {
  if (!b) return;
  release(b);
  delete b;
}

void ce::batch_detach(ce_batch* b, ce_sim* s) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& m : b->members)
    if (m == s) m = nullptr;
  b->broken = true;
}

extern "C" {

int ce_batch_create(ce_sim* const* sims, int n, int sweep_len, int ctas_per_sm, void* stream, ce_batch** out) {
  ce::set_last_error("");
  if (!out) return bfail(CE_EINVAL, "ce_batch_create: out is NULL");
  *out = nullptr;
  if (!sims || n < 1) return bfail(CE_EINVAL, "ce_batch_create: need at least one simulation");
  if (sweep_len < 0 || sweep_len > 4096) return bfail(CE_EINVAL, "ce_batch_create: sweep_len must be 0..4096");
  if (ctas_per_sm < 0 || ctas_per_sm > 8) return bfail(CE_EINVAL, "ce_batch_create: ctas_per_sm must be 0..8");
  const ce_sim* s0 = sims[0];
  if (!s0) return bfail(CE_EINVAL, "ce_batch_create: NULL member");
  for (int k = 0; k < n; ++k) {
    const ce_sim* s = sims[k];
    if (!s) return bfail(CE_EINVAL, "ce_batch_create: NULL member");
    if (s->batch) return bfail(CE_ESTATE, "ce_batch_create: a member already belongs to a batch");
    if (!s->have_state) return bfail(CE_ESTATE, "ce_batch_create: a member has no fields set");
    if (s->prec != s0->prec || s->nf != s0->nf)
      return bfail(CE_EINVAL, "ce_batch_create: members must share precision and number of fields");
    if (s->device != s0->device) return bfail(CE_EINVAL, "ce_batch_create: members must live on one device");
    const int vx = s->prec == CE_F32 ? 4 : 2;
    if (s->N % vx != 0)
      return bfail(CE_EINVAL, "ce_batch_create: N must be a multiple of 4 (FP32) or 2 (FP64) in a batch");
    for (int j = 0; j < k; ++j)
      if (sims[j] == s) return bfail(CE_EINVAL, "ce_batch_create: a simulation is listed twice");
  }
  cudaError_t e = cudaSetDevice(s0->device);
  if (e != cudaSuccess) return bcuda(e, "ce_batch_create");
  ce_batch* b = new (std::nothrow) ce_batch();
  if (!b) return bfail(CE_ENOMEM, "ce_batch_create: host allocation");
  b->members.assign(sims, sims + n);
  b->prec = s0->prec;
  b->nf = s0->nf;
  b->device = s0->device;
  b->sweep_len = sweep_len > 0 ? sweep_len : 128;
  b->ctas_per_sm = ctas_per_sm;
  for (ce_sim* s : b->members) {
    e = cudaStreamSynchronize(s->stream);   // members' own queued work finishes first
    if (e != cudaSuccess) {
      delete b;
      return bcuda(e, "ce_batch_create: member sync");
    }
    b->sites += s->S;
  }
  if (stream) {
    b->stream = static_cast<cudaStream_t>(stream);
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return bcuda(e, "ce_batch_create: stream");
    }
    b->own_stream = true;
  }
  e = cudaMalloc(&b->d_queue, sizeof(unsigned int) * (2 + n));
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned int) * (2 + n), b->stream);
  if (e != cudaSuccess) {
    release(b);
    delete b;
    return bcuda(e, "ce_batch_create: scratch");
  }
  b->d_done = b->d_queue + 2;
  int rc = b->prec == CE_F32 ? upload_tables<float>(b) : upload_tables<double>(b);
  if (rc != CE_OK) {
    release(b);
    delete b;
    return rc;
  }
  int per_sm = 0, sms = 0;
  e = batch_prepare(b->prec, b->nf, &per_sm);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess && b->ctas_per_sm > 0) per_sm = std::min(per_sm, b->ctas_per_sm);
  if (e != cudaSuccess || per_sm < 1) {
    release(b);
    delete b;
    return bcuda(e != cudaSuccess ? e : cudaErrorInvalidConfiguration, "ce_batch_create: occupancy");
  }
  b->blocks = std::max(1, std::min(per_sm * sms, b->n_items));
  if (b->n1d > 0 && b->n_items > 0) {
    e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      release(b);
      delete b;
      return bcuda(e, "ce_batch_create: side stream");
    }
  }
  for (ce_sim* s : b->members) s->batch = b;
  *out = b;
  return CE_OK;
}

int ce_batch_step(ce_batch* b, int64_t n) {
  ce::set_last_error("");
  if (!b) return bfail(CE_EINVAL, "ce_batch_step: batch is NULL");
  if (n < 0) return bfail(CE_EINVAL, "ce_batch_step: n must be >= 0");
  if (b->broken) return bfail(CE_ESTATE, "ce_batch_step: a member was freed; free and rebuild the batch");
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bcuda(e, "ce_batch_step");
  while (n >= ce::kBatchGraphSteps && b->graphs_ok) {
    e = ensure_batch_graph(b, b->par);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->graphs_ok = false;
      break;
    }
    e = cudaGraphLaunch(b->graph[b->par], b->stream);
    if (e != cudaSuccess) return bcuda(e, "ce_batch_step: graph launch");
    advance_members(b, ce::kBatchGraphSteps);
    n -= ce::kBatchGraphSteps;
  }
  if (n > 0) {
    e = fork_side(b);
    if (e != cudaSuccess) return bcuda(e, "ce_batch_step: fork");
    for (int64_t k = 0; k < n; ++k) {
      e = launch_batch(b, b->par);
      if (e != cudaSuccess) return bcuda(e, "ce_batch_step: launch");
      b->par ^= 1;
      advance_members(b, 1);
    }
    e = join_side(b);
    if (e != cudaSuccess) return bcuda(e, "ce_batch_step: join");
  }
  return CE_OK;
}

int ce_batch_synchronize(ce_batch* b) {
  ce::set_last_error("");
  if (!b) return bfail(CE_EINVAL, "ce_batch_synchronize: batch is NULL");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "ce_batch_synchronize");
  for (ce_sim* s : b->members) {
    if (!s) continue;
    int st = 0;
    e = cudaMemcpy(&st, &s->aux->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(e, "ce_batch_synchronize: status");
    if (st != CE_OK) return bfail(st, "ce_batch_synchronize: a member reported non-finite sums or a timeout");
  }
  return CE_OK;
}

int ce_batch_status(ce_batch* b, int* status, int n) {
  ce::set_last_error("");
  if (!b || !status) return bfail(CE_EINVAL, "ce_batch_status: NULL argument");
  if (n < (int)b->members.size()) return bfail(CE_EINVAL, "ce_batch_status: status array shorter than the batch");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "ce_batch_status");
  for (size_t k = 0; k < b->members.size(); ++k) {
    status[k] = CE_OK;
    if (!b->members[k]) continue;
    e = cudaMemcpy(&status[k], &b->members[k]->aux->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(e, "ce_batch_status: status");
  }
  return CE_OK;
}

int ce_batch_info(const ce_batch* b, int* members, int* items, int* blocks, int64_t* sites) {
  if (!b || !members || !items || !blocks || !sites) return bfail(CE_EINVAL, "ce_batch_info: NULL argument");
  *members = (int)b->members.size();
  *items = b->n_units;
  *blocks = b->blocks;
  *sites = b->sites;
  return CE_OK;
}

void ce_batch_free(ce_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  for (ce_sim* s : b->members)
    if (s) s->batch = nullptr;
  release(b);
  delete b;
}

}  // extern "C"
