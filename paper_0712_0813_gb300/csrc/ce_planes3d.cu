// ce_planes3d.cu -- the 3D step for any side N: a block owns a 64 x 8 column
// of sites and sweeps a chunk of z-planes, with plain coalesced loads (no
// alignment needed, so odd sides work), each site's drifted g formed once per
// plane in shared memory, and z-neighbours carried in registers.
//
// Per site the arithmetic is the generic kernel's (arXiv:0712.0813 Sec. III
// staggered leapfrog, fused: v = w + c f, g = f + dt v, lap g from the 2d
// nearest neighbours in the order x, y, z, w_out = v + dt (lap g - dV/df(g)),
// f_out = g), so the fields agree with k_step_generic bit for bit; only the
// global sums are added in another order.
//
// Block: 10 warps over a tile of 32 SX x 8 sites.  Warps 1..8 own the tile
// rows y0 .. y0 + 7, lane l the sites x0 + l + 32 h, h < SX.  SX = 2 on large
// lattices (from side 192: the per-plane costs -- offsets, the barrier, the
// loop -- are shared by two sites, and the second site's loads and stores use
// immediate offsets; 383^3: 432 -> 413 us), SX = 1 below (more blocks: 64^3
// 13.1 against 16.8 us).  Warp 0
// computes the y-halo row y0 - 1 and warp 9 the row after the last tile row
// (both mod N), so every g in the staged plane is computed once by one thread.
// Warp 0 also computes the x-halo sites: lane l < 16 the site x0 - 1 of tile
// row l, lane 16 + l the site x0 + nx of tile row l (mod N; nx is the tile's
// width), which keeps the tile warps' instruction stream free of halo work.
//
// Loads: every thread copies the f and w values it needs (its own sites, and
// its x-halo site) with 4- or 8-byte cp.async into a shared-memory ring
// D planes deep, D - 1 planes ahead of the plane it forms (D = 4 for FP32 with
// up to 2 fields; fewer where the ring would not fit); only the thread itself
// reads those slots, so the ring needs no barrier, and the copies in flight
// hold no registers (the latency of HBM needs ~40 KB in flight per SM).  A
// plane's g goes into one of three g buffers; the single block barrier per
// plane publishes it, and three buffers make that one barrier enough (a buffer
// is rewritten two planes after it was last read).  The z-chunk covers planes
// z0 .. z1 - 1 and stages z0 - 1 and z1 as well.
#include <cstdint>

#include "ce_device.cuh"
#include "ce_internal.h"
#include "ce_tma.cuh"

namespace ce {
namespace {

constexpr int kPlaneRows = 8;                 // tile rows per block
constexpr int kPlaneWarps = kPlaneRows + 2;   // plus the two y-halo warps
constexpr int kPlaneThreads = 32 * kPlaneWarps;
// staged columns: x-halo, the 32 SX tile columns, x-halo
template <int SX>
struct Tile {
  static constexpr int X = 32 * SX;
  static constexpr int cols = X + 2;
  static constexpr int cells = (kPlaneRows + 2) * cols;
};

// planes of f, w in the copy ring: the ring and three g buffers fit the SM's
// shared memory for every storage type and field count
template <typename T, int NF>
struct RingDepth {
  static constexpr int value = sizeof(T) * NF <= 8 ? 4 : (sizeof(T) * NF <= 16 ? 3 : 2);
};

// dynamic shared memory: 3 g buffers of NF planes, then the copy ring
template <typename T, int NF, int SX>
constexpr size_t planes_smem() {
  return sizeof(T) * (size_t)Tile<SX>::cells * NF * (3 + 2 * RingDepth<T, NF>::value);
}

template <typename T, int NF, int SX>
__global__ void __launch_bounds__(kPlaneThreads) k_step_planes(const StepArgs<T> p, int zlen) {
  constexpr int D = RingDepth<T, NF>::value;
  constexpr int kTileX = Tile<SX>::X, kPlaneCols = Tile<SX>::cols, kPlaneCells = Tile<SX>::cells;
  extern __shared__ __align__(16) unsigned char planes_smem_dyn[];
  T* const sg = reinterpret_cast<T*>(planes_smem_dyn);             // [3][NF][rows + 2][cols]
  T* const ring = sg + 3 * NF * kPlaneCells;                        // [D][NF][f, w][rows + 2][cols]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t N = p.N, NN = N * N;
  const int x0 = blockIdx.x * kTileX, y0 = blockIdx.y * kPlaneRows;
  const int nx = (int)min((int64_t)kTileX, N - x0), ny = (int)min((int64_t)kPlaneRows, N - y0);
  const int z0 = blockIdx.z * zlen;
  const int z1 = (int)min((int64_t)z0 + zlen, N);
  // staged row r of this warp: 0 = row y0 - 1, 1 .. ny = tile rows, ny + 1 = the row after them
  const int r = warp == kPlaneWarps - 1 ? ny + 1 : warp;
  const bool row_on = warp == 0 || warp == kPlaneWarps - 1 || warp <= ny;
  const bool tile_row = warp >= 1 && warp <= ny;
  // sites h < SX of this lane: x0 + lane + 32 h, inside the tile when < nx
  bool act[SX], upd_site[SX];
#pragma unroll
  for (int h = 0; h < SX; ++h) {
    act[h] = row_on && lane + 32 * h < nx;         // forms a g each plane
    upd_site[h] = tile_row && lane + 32 * h < nx;  // updates the site
  }
  const auto wrap = [&](int64_t v) { return v < 0 ? v + N : (v >= N ? v - N : v); };
  const int64_t yrow = wrap((int64_t)y0 - 1 + r);
  const int64_t own = yrow * N + x0 + lane;                 // offset inside a plane of site 0
  // x-halo site of this lane (warp 0 only): staged row hr = 1 + (lane mod 16),
  // column 0 (x0 - 1) for lanes 0..15, column nx + 1 (x0 + nx) for lanes 16..31
  static_assert(kPlaneRows <= 16, "warp 0 holds one x-halo site per tile row and side");
  const int hr = 1 + (lane & 15);
  const bool halo = warp == 0 && hr <= ny;
  const int hcol = lane < 16 ? 0 : nx + 1;
  const int64_t hoff = wrap((int64_t)y0 - 1 + hr) * N + (lane < 16 ? wrap((int64_t)x0 - 1) : wrap((int64_t)x0 + nx));
  const int cell = r * kPlaneCols + lane + 1, hcell = hr * kPlaneCols + hcol;   // site h: cell + 32 h

  const T c = (T)p.sc_in->c;
  const T dd = p.dt_drift, kk = p.dt_kick, idx2 = p.inv_dx2;
  const T q[3] = {p.q[0], p.q[1], p.q[2]};
  const int n = z1 - z0 + 2;                                // staged planes z0 - 1 .. z1

  // per-thread column pointers; the plane offset advances by N^2 per staged
  // plane and wraps once (periodic z)
  const T* fo[NF];
  const T* wo[NF];
  const T* fh[NF];
  const T* wh[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    fo[i] = p.f_in[i] + own;
    wo[i] = p.w_in[i] + own;
    fh[i] = p.f_in[i] + hoff;
    wh[i] = p.w_in[i] + hoff;
  }
  int64_t zoff = (int64_t)(z0 == 0 ? N - 1 : z0 - 1) * NN;   // offset of the next plane to copy
  const int64_t wrap_at = (N - 1) * NN;
  // copy the next staged plane into ring slot `slot`, as one commit group
  // (an empty group past the chunk keeps the group count uniform)
  const auto issue = [&](int slot, bool any) {
    if (any) {
      T* rs = ring + (size_t)slot * NF * 2 * kPlaneCells;
#pragma unroll
      for (int i = 0; i < NF; ++i) {
#pragma unroll
        for (int h = 0; h < SX; ++h)
          if (act[h]) {
            cp_small<sizeof(T)>(rs + (2 * i) * kPlaneCells + cell + 32 * h, fo[i] + zoff + 32 * h);
            cp_small<sizeof(T)>(rs + (2 * i + 1) * kPlaneCells + cell + 32 * h, wo[i] + zoff + 32 * h);
          }
        if (halo) {
          cp_small<sizeof(T)>(rs + (2 * i) * kPlaneCells + hcell, fh[i] + zoff);
          cp_small<sizeof(T)>(rs + (2 * i + 1) * kPlaneCells + hcell, wh[i] + zoff);
        }
      }
      zoff = zoff == wrap_at ? 0 : zoff + NN;
    }
    cp_commit();
  };

  // three register sets: R[k] holds g (and v) of the staged planes j = k mod 3
  T g0[NF][SX], g1[NF][SX], g2[NF][SX], v0[NF][SX], v1[NF][SX], v2[NF][SX];
#pragma unroll
  for (int i = 0; i < NF; ++i)
#pragma unroll
    for (int h = 0; h < SX; ++h) g0[i][h] = g1[i][h] = g2[i][h] = v0[i][h] = v1[i][h] = v2[i][h] = T(0);
  // two-level sums in T, converted to FP64 once per thread (see k_step_generic)
  T g2acc = T(0), vacc = T(0), g2loc = T(0), vloc = T(0);
  int since_flush = 0;
  int64_t upd = (int64_t)z0 * NN + own;                     // output offset of the next updated plane

  // staged plane j: form its g from ring slot j mod D into g buffer `form`
  // (j mod 3) and gn, copy plane j + D - 1 into its slot (that of plane j - 1,
  // which this thread read in the previous stage), then (j >= 2) update plane
  // j - 1 from g buffer `read` ((j - 1) mod 3) with z-neighbours gm (plane
  // j - 2) and gn (plane j), own g gc and v vc (plane j - 1)
  const auto stage = [&](int j, T* form, const T* read, T (&gn)[NF][SX], T (&vn)[NF][SX], const T (&gm)[NF][SX],
                         const T (&gc)[NF][SX], const T (&vc)[NF][SX]) {
    cp_wait<D - 2>();                                       // this thread's copies of plane j have landed
    const T* rs = ring + (size_t)(j % D) * NF * 2 * kPlaneCells;
#pragma unroll
    for (int i = 0; i < NF; ++i) {
#pragma unroll
      for (int h = 0; h < SX; ++h)
        if (act[h]) {
          const T f = rs[(2 * i) * kPlaneCells + cell + 32 * h], w = rs[(2 * i + 1) * kPlaneCells + cell + 32 * h];
          vn[i][h] = fmaT(c, f, w);
          gn[i][h] = fmaT(dd, vn[i][h], f);
          form[i * kPlaneCells + cell + 32 * h] = gn[i][h];
        }
      if (halo) {
        const T f = rs[(2 * i) * kPlaneCells + hcell], w = rs[(2 * i + 1) * kPlaneCells + hcell];
        form[i * kPlaneCells + hcell] = fmaT(dd, fmaT(c, f, w), f);
      }
    }
    issue((j + D - 1) % D, j + D - 1 < n);                  // the slot of plane j - 1, read last stage
    __syncthreads();
    if (j < 2 || !tile_row) return;
#pragma unroll
    for (int h = 0; h < SX; ++h) {
      if (!upd_site[h]) continue;
      T lap[NF], gs[NF];
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        const T* rd = read + i * kPlaneCells + cell + 32 * h;
        const T g = gc[i][h];
        T acc = T(0);
        {
          const T xp = rd[1], xm = rd[-1];
          acc += (xp + xm) - T(2) * g;
          const T df = xp - g;
          g2loc = fmaT(df, df, g2loc);
        }
        {
          const T yp = rd[kPlaneCols], ym = rd[-kPlaneCols];
          acc += (yp + ym) - T(2) * g;
          const T df = yp - g;
          g2loc = fmaT(df, df, g2loc);
        }
        {
          acc += (gn[i][h] + gm[i][h]) - T(2) * g;
          const T df = gn[i][h] - g;
          g2loc = fmaT(df, df, g2loc);
        }
        lap[i] = acc * idx2;
        gs[i] = g;
      }
      T dv[NF], vs;
      model_dv<T, NF>(gs, q, dv, vs);
      vloc += vs;
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        __stcs(p.w_out[i] + upd + 32 * h, fmaT(kk, lap[i] - dv[i], vc[i][h]));
        __stcs(p.f_out[i] + upd + 32 * h, gs[i]);
      }
      ++since_flush;
    }
    upd += NN;   // the chunk's planes z0 .. z1 - 1 do not wrap
    if (since_flush >= 16) {
      g2acc += g2loc;
      vacc += vloc;
      g2loc = T(0);
      vloc = T(0);
      since_flush = 0;
    }
  };
#pragma unroll
  for (int k = 0; k < D - 1; ++k) issue(k, k < n);
  T* const b0 = sg;
  T* const b1 = sg + NF * kPlaneCells;
  T* const b2 = sg + 2 * NF * kPlaneCells;
  for (int j = 0; j < n; j += 3) {
    stage(j, b0, b2, g0, v0, g1, g2, v2);
    if (j + 1 < n) stage(j + 1, b1, b0, g1, v1, g2, g0, v0);
    if (j + 2 < n) stage(j + 2, b2, b1, g2, v2, g0, g1, v1);
  }
  cp_wait<0>();
  if (p.update_scalars) finish_step_block(p, (double)g2acc + (double)g2loc, (double)vacc + (double)vloc);
}

template <typename T, int NF>
cudaError_t launch_nf(const StepArgs<T>& a, const PlanesPlan& pl, cudaStream_t st) {
  if (pl.sx == 2)
    k_step_planes<T, NF, 2><<<dim3(pl.gx, pl.gy, pl.gz), kPlaneThreads, planes_smem<T, NF, 2>(), st>>>(a, pl.zlen);
  else
    k_step_planes<T, NF, 1><<<dim3(pl.gx, pl.gy, pl.gz), kPlaneThreads, planes_smem<T, NF, 1>(), st>>>(a, pl.zlen);
  return cudaGetLastError();
}

// Raise the kernel's dynamic shared-memory limit (FP64 with 4 fields needs
// ~120 KB at SX = 1) and report how many blocks fit an SM.
template <typename T, int NF, int SX>
int blocks_per_sm() {
  const void* k = (const void*)&k_step_planes<T, NF, SX>;
  int n = 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)planes_smem<T, NF, SX>()) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kPlaneThreads, planes_smem<T, NF, SX>()) !=
          cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n < 1 ? 1 : n;
}

template <typename T, int SX>
int blocks_per_sm_nf(int nf) {
  return nf == 1 ? blocks_per_sm<T, 1, SX>() : nf == 2 ? blocks_per_sm<T, 2, SX>()
       : nf == 3 ? blocks_per_sm<T, 3, SX>() : blocks_per_sm<T, 4, SX>();
}

constexpr int64_t kTwoSitesMinN = 192;   // sides from which each lane takes two sites

}  // namespace

// Grid of the plane-sweep kernel: 32 SX x 8 columns of sites, z split into
// chunks so that about two waves of resident blocks are busy, with chunks of
// at least 8 planes (each chunk stages 2 halo planes besides its own).
PlanesPlan planes_plan(int64_t N, int nf, int prec, int sms) {
  PlanesPlan pl{};
  pl.sx = N >= kTwoSitesMinN ? 2 : 1;
  pl.gx = (int)((N + 32 * pl.sx - 1) / (32 * pl.sx));
  pl.gy = (int)((N + kPlaneRows - 1) / kPlaneRows);
  int per_sm;
  if (prec == CE_F32) per_sm = pl.sx == 2 ? blocks_per_sm_nf<float, 2>(nf) : blocks_per_sm_nf<float, 1>(nf);
  else per_sm = pl.sx == 2 ? blocks_per_sm_nf<double, 2>(nf) : blocks_per_sm_nf<double, 1>(nf);
  const int64_t cols = (int64_t)pl.gx * pl.gy;
  const int64_t want = std::max<int64_t>(1, (2LL * per_sm * sms + cols - 1) / cols);
  const int64_t gz = std::max<int64_t>(1, std::min<int64_t>(want, N / 8));
  pl.zlen = (int)((N + gz - 1) / gz);
  pl.gz = (int)((N + pl.zlen - 1) / pl.zlen);
  return pl;
}

template <typename T>
cudaError_t launch_step_planes(const StepArgs<T>& a, const PlanesPlan& pl, cudaStream_t st) {
  switch (a.nf) {
    case 1: return launch_nf<T, 1>(a, pl, st);
    case 2: return launch_nf<T, 2>(a, pl, st);
    case 3: return launch_nf<T, 3>(a, pl, st);
    default: return launch_nf<T, 4>(a, pl, st);
  }
}
template cudaError_t launch_step_planes<float>(const StepArgs<float>&, const PlanesPlan&, cudaStream_t);
template cudaError_t launch_step_planes<double>(const StepArgs<double>&, const PlanesPlan&, cudaStream_t);

}  // namespace ce
