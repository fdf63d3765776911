// ce_cols3d.cu -- the 3D step for any side N with the neighbours in registers:
// each warp owns a strip of 30 x-sites by TY rows and sweeps a chunk of z, with
// plain coalesced loads (no alignment needed, so odd sides work), no shared
// memory and no block barrier in the sweep.
//
// Per site the arithmetic is the generic kernel's (arXiv:0712.0813 Sec. III
// staggered leapfrog, fused: v = w + c f, g = f + dt v, lap g from the 2d
// nearest neighbours in the order x, y, z, w_out = v + dt (lap g - dV/df(g)),
// f_out = g), so the fields agree with k_step_generic bit for bit; only the
// global sums are added in another order.
//
// Warp layout.  Lane l holds the column x0 - 1 + l (mod N) of the strip, for
// the TY + 2 rows y0 - 1 .. y0 + TY (mod N); lanes 1 .. nx (nx <= 30) update
// their sites, lanes 0 and nx + 1 hold the strip's x-halo (lanes past nx + 1
// repeat lane nx + 1's column), so the x-neighbours of every updated site come
// from the adjacent lanes by shuffles and no lane loads anything twice.  The
// y-neighbours are the lane's own registers one row up or down; the y-halo
// rows are the own rows of the neighbouring row group, loaded by another warp
// at about the same time (L2).  Along z each lane keeps g of three planes, the
// one being updated and its two z-neighbours, in registers, and the loads of
// the plane after them in flight.  Neighbouring z-chunks sweep in opposite
// directions, so the two chunks that share a boundary read its planes at about
// the same time.
//
// TY (rows per lane), ColRows below: FP32 6 rows for 1-2 fields (4 below side
// 160), 3 / 2 for 3 / 4 fields; FP64 4 rows for 1 field, 2 for more.  Loop
// unrolled by 3 so that the three g buffers keep static register roles.
#include <cstdint>

#include "ce_device.cuh"
#include "ce_internal.h"
#include "ce_plan.h"

namespace ce {
namespace {

constexpr int kColWarps = 4;
constexpr int kColThreads = 32 * kColWarps;
constexpr int kStrip = 30;   // sites a warp updates along x

// Rows per lane: registers per thread near the 168 that 3 blocks of 128
// threads per SM allow.  Lattices below side 160 take fewer rows (more warps
// per plane: they are bound by the latency of a warp's sweep, not by HBM).
template <typename T, int NF, bool NARROW>
struct ColRows {
  static constexpr int wide = sizeof(T) == 4 ? (NF <= 2 ? 6 : (NF == 3 ? 3 : 2)) : (NF == 1 ? 4 : 2);
  static constexpr int value = NARROW ? (wide >= 6 ? 4 : (wide == 3 ? 2 : wide)) : wide;
};
constexpr int64_t kNarrowBelow = 160;

template <typename T, int NF, int TY, int MB = 3>
__global__ void __launch_bounds__(kColThreads, MB) k_step_cols(const StepArgs<T> p, int nstrips, int ngroups,
                                                              int zlen) {
  constexpr int R = TY + 2;   // rows a lane holds: y0 - 1 .. y0 + TY
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t N = p.N, NN = N * N;
  const int64_t wg = (int64_t)blockIdx.x * kColWarps + warp;
  T g2acc = T(0), vacc = T(0), g2loc = T(0), vloc = T(0);   // two-level sums (see k_step_generic)
  if (wg < (int64_t)nstrips * ngroups) {
    const int strip = (int)(wg % nstrips), grp = (int)(wg / nstrips);
    const int64_t x0 = (int64_t)strip * kStrip;
    const int nx = (int)min((int64_t)kStrip, N - x0);
    const int y0 = grp * TY;
    const int ny = (int)min((int64_t)TY, N - y0);
    const int z0 = blockIdx.y * zlen;
    const int z1 = (int)min((int64_t)z0 + zlen, N);
    const int np = z1 - z0 + 2;                    // planes z0 - 1 .. z1
    const bool down = (blockIdx.y & 1u) != 0;
    int64_t xs = x0 - 1 + min(lane, nx + 1);
    xs = xs < 0 ? xs + N : (xs >= N ? xs - N : xs);
    const bool site = lane >= 1 && lane <= nx;
    int ry[R];                                     // offsets of the lane's rows in a plane, plus its column
#pragma unroll
    for (int k = 0; k < R; ++k) {
      int y = y0 - 1 + k;
      y = y < 0 ? y + (int)N : y;
      y = y >= N ? y - (int)N : y;
      y = y >= N ? y % (int)N : y;                 // N < TY + 1: several wraps
      ry[k] = y * (int)N + (int)xs;                // N^2 < 2^31 (3D sides up to 46340)
    }
    const T c = (T)p.sc_in->c;
    const T dd = p.dt_drift, kk = p.dt_kick, idx2 = p.inv_dx2;
    const T q[3] = {p.q[0], p.q[1], p.q[2]};
    // plane k of the sweep: z0 - 1 + k upwards, z1 - k downwards (mod N)
    const auto plane_off = [&](int k) -> int64_t {
      int64_t z = down ? (int64_t)z1 - k : (int64_t)z0 - 1 + k;
      z = z < 0 ? z + N : (z >= N ? z - N : z);
      return z * NN;
    };
    T lf[NF][R], lw[NF][R];                        // loads in flight: the next plane to form
    const auto issue = [&](int k) {
      const int64_t po = plane_off(k);
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        const T* fi = p.f_in[i] + po;
        const T* wi = p.w_in[i] + po;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          lf[i][r] = __ldg(fi + ry[r]);
          lw[i][r] = __ldg(wi + ry[r]);
        }
      }
    };
    // g of the loaded plane on every row, v on the own rows
    const auto form = [&](T (&g)[NF][R], T (&v)[NF][TY]) {
#pragma unroll
      for (int i = 0; i < NF; ++i) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const T vr = fmaT(c, lf[i][r], lw[i][r]);
          g[i][r] = fmaT(dd, vr, lf[i][r]);
          if (r >= 1 && r <= TY) v[i][r - 1] = vr;
        }
      }
    };
    int since_flush = 0;
    // update sweep plane k (1 .. np - 2): gP / gN are the planes before and
    // after it in the sweep, so z + 1 is gN upwards and gP downwards
    const auto update = [&](int k, const T (&gP)[NF][R], const T (&gC)[NF][R], const T (&gN)[NF][R],
                            const T (&vC)[NF][TY]) {
      const int64_t po = plane_off(k);
#pragma unroll
      for (int j = 0; j < TY; ++j) {
        if (j >= ny) break;
        const int r = j + 1;
        T xms[NF], xps[NF];
#pragma unroll
        for (int i = 0; i < NF; ++i) {   // every lane takes part in the shuffles
          xms[i] = __shfl_up_sync(0xffffffffu, gC[i][r], 1);
          xps[i] = __shfl_down_sync(0xffffffffu, gC[i][r], 1);
        }
        if (site) {
          T lap[NF], gs[NF];
#pragma unroll
          for (int i = 0; i < NF; ++i) {
            const T g = gC[i][r];
            const T zp = down ? gP[i][r] : gN[i][r], zm = down ? gN[i][r] : gP[i][r];
            T acc = T(0);
            acc += (xps[i] + xms[i]) - T(2) * g;
            T df = xps[i] - g;
            g2loc = fmaT(df, df, g2loc);
            acc += (gC[i][r + 1] + gC[i][r - 1]) - T(2) * g;
            df = gC[i][r + 1] - g;
            g2loc = fmaT(df, df, g2loc);
            acc += (zp + zm) - T(2) * g;
            df = zp - g;
            g2loc = fmaT(df, df, g2loc);
            lap[i] = acc * idx2;
            gs[i] = g;
          }
          T dv[NF], vs;
          model_dv<T, NF>(gs, q, dv, vs);
          vloc += vs;
          const int64_t o = po + ry[r];
#pragma unroll
          for (int i = 0; i < NF; ++i) {
            __stcs(p.w_out[i] + o, fmaT(kk, lap[i] - dv[i], vC[i][j]));
            __stcs(p.f_out[i] + o, gs[i]);
          }
        }
      }
      since_flush += ny;
      if (since_flush >= 16) {
        g2acc += g2loc;
        vacc += vloc;
        g2loc = T(0);
        vloc = T(0);
        since_flush = 0;
      }
    };
    // plane k of the sweep goes into buffer k % 3
    T gA[NF][R], gB[NF][R], gC3[NF][R];
    T vA[NF][TY], vB[NF][TY], vC3[NF][TY];
    const auto stage = [&](int k, const T (&gP)[NF][R], const T (&gC)[NF][R], T (&gN)[NF][R],
                           const T (&vC)[NF][TY], T (&vN)[NF][TY]) {
      form(gN, vN);                  // plane k + 1, loaded one stage ago
      if (k + 2 < np) issue(k + 2);
      update(k, gP, gC, gN, vC);
    };
    issue(0);
    form(gA, vA);
    issue(1);
    form(gB, vB);
    issue(2);
    int k = 1;
    for (; k + 2 <= np - 2; k += 3) {
      stage(k, gA, gB, gC3, vB, vC3);
      stage(k + 1, gB, gC3, gA, vC3, vA);
      stage(k + 2, gC3, gA, gB, vA, vB);
    }
    if (k <= np - 2) {
      stage(k, gA, gB, gC3, vB, vC3);
      ++k;
    }
    if (k <= np - 2) stage(k, gB, gC3, gA, vC3, vA);
  }
  if (p.update_scalars) finish_step_block(p, (double)g2acc + (double)g2loc, (double)vacc + (double)vloc);
}

template <typename T, int NF>
cudaError_t launch_nf(const StepArgs<T>& a, const ColsPlan& pl, cudaStream_t st) {
  const dim3 grid(pl.gx, pl.gz);
  if (pl.ty == ColRows<T, NF, false>::value)
    k_step_cols<T, NF, ColRows<T, NF, false>::value><<<grid, kColThreads, 0, st>>>(a, pl.nstrips, pl.ngroups, pl.zlen);
  else
    k_step_cols<T, NF, ColRows<T, NF, true>::value><<<grid, kColThreads, 0, st>>>(a, pl.nstrips, pl.ngroups, pl.zlen);
  return cudaGetLastError();
}

template <typename T, int NF>
void rows_and_occupancy(bool narrow, int& ty, int& per_sm) {
  const void* k;
  if (narrow) {
    ty = ColRows<T, NF, true>::value;
    k = (const void*)k_step_cols<T, NF, ColRows<T, NF, true>::value>;
  } else {
    ty = ColRows<T, NF, false>::value;
    k = (const void*)k_step_cols<T, NF, ColRows<T, NF, false>::value>;
  }
  per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kColThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  per_sm = std::max(per_sm, 1);
}

template <typename T>
void rows_and_occupancy_nf(int nf, bool narrow, int& ty, int& per_sm) {
  switch (nf) {
    case 1: rows_and_occupancy<T, 1>(narrow, ty, per_sm); break;
    case 2: rows_and_occupancy<T, 2>(narrow, ty, per_sm); break;
    case 3: rows_and_occupancy<T, 3>(narrow, ty, per_sm); break;
    default: rows_and_occupancy<T, 4>(narrow, ty, per_sm); break;
  }
}

}  // namespace

// Grid of the column kernel: warps over (strip, row group), 4 per block, and
// the z-chunk length of the wave model (plan::wave_chunk_length: chunks of at
// least 4 planes, each costing 5 more for its halo planes and start-up).
ColsPlan cols_plan(int64_t N, int nf, int prec, int sms) {
  ColsPlan pl{};
  int per_sm = 1;
  if (prec == CE_F32) rows_and_occupancy_nf<float>(nf, N < kNarrowBelow, pl.ty, per_sm);
  else rows_and_occupancy_nf<double>(nf, N < kNarrowBelow, pl.ty, per_sm);
  pl.nstrips = (int)((N + kStrip - 1) / kStrip);
  pl.ngroups = (int)((N + pl.ty - 1) / pl.ty);
  const int64_t warps = (int64_t)pl.nstrips * pl.ngroups;
  pl.gx = (int)((warps + kColWarps - 1) / kColWarps);
  pl.zlen = plan::wave_chunk_length(N, pl.gx, (int64_t)per_sm * sms, 4, 5.0);   // ce_plan.h
  pl.gz = (int)((N + pl.zlen - 1) / pl.zlen);
  return pl;
}

template <typename T>
cudaError_t launch_step_cols(const StepArgs<T>& a, const ColsPlan& pl, cudaStream_t st) {
  switch (a.nf) {
    case 1: return launch_nf<T, 1>(a, pl, st);
    case 2: return launch_nf<T, 2>(a, pl, st);
    case 3: return launch_nf<T, 3>(a, pl, st);
    default: return launch_nf<T, 4>(a, pl, st);
  }
}
template cudaError_t launch_step_cols<float>(const StepArgs<float>&, const ColsPlan&, cudaStream_t);
template cudaError_t launch_step_cols<double>(const StepArgs<double>&, const ColsPlan&, cudaStream_t);

}  // namespace ce
