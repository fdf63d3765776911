// ce_lines2d.cu -- the 2D step for any side N: each warp sweeps a strip of 30
// x-sites along a chunk of rows y, with plain coalesced loads (no alignment
// needed, so odd sides work), y-neighbours carried in registers and
// x-neighbours exchanged by warp shuffles: no shared memory, no block barrier.
//
// Per site the arithmetic is the generic kernel's (arXiv:0712.0813 Sec. III
// staggered leapfrog, fused: v = w + c f, g = f + dt v, lap g from the 2d
// nearest neighbours in the order x, y, w_out = v + dt (lap g - dV/df(g)),
// f_out = g), so the fields agree with k_step_generic bit for bit; only the
// global sums are added in another order.
//
// Warp w of block b owns the strip x0 = 30 (8 b.x + w) .. x0 + nx - 1 (nx <= 30)
// and the rows y0 .. y1 - 1 of chunk b.y, and forms g on the rows y0 - 1 .. y1
// (mod N).  Lane l holds the column x0 - 1 + l (mod N): lanes 1 .. nx update
// their sites, lanes 0 and nx + 1 hold the strip's x-halo (lanes past nx + 1
// repeat lane nx + 1's column), so one load instruction per field and array
// brings a row with its halo and the shuffles give every updated site both
// x-neighbours.  Each lane keeps the loads of the next DL rows in flight in a
// ring of registers (DL = 8 / 6 / 4 for 1 / 2 / 3-4 fields): 2-3 KB per warp,
// which the latency of HBM needs.  Neighbouring chunks sweep in opposite directions, so
// the two chunks that share a boundary row read it at about the same time.
#include <cstdint>

#include "ce_device.cuh"
#include "ce_internal.h"
#include "ce_plan.h"

namespace ce {
namespace {

constexpr int kLineWarps = 8;
constexpr int kLineThreads = 32 * kLineWarps;
constexpr int kStrip = 30;   // sites a warp updates along x

// rows of loads in flight per lane (6001^2, 2 fields: 4 rows 229.0 us, 6 rows
// 223.8, 8 rows 228.9, the last at 3 instead of 4 blocks per SM; 16001^2: 1642,
// 1497, 1541 us)
template <int NF>
struct LineDepth {
  static constexpr int value = NF == 1 ? 8 : (NF == 2 ? 6 : 4);
};

template <typename T, int NF, int DL>
__global__ void __launch_bounds__(kLineThreads) k_step_lines(const StepArgs<T> p, int nstrips, int ylen) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t N = p.N;
  const int64_t wg = (int64_t)blockIdx.x * kLineWarps + warp;
  T g2acc = T(0), vacc = T(0), g2loc = T(0), vloc = T(0);   // two-level sums (see k_step_generic)
  if (wg < nstrips) {
    const int64_t x0 = wg * kStrip;
    const int nx = (int)min((int64_t)kStrip, N - x0);
    int64_t xs = x0 - 1 + min(lane, nx + 1);
    xs = xs < 0 ? xs + N : (xs >= N ? xs - N : xs);
    const bool site = lane >= 1 && lane <= nx;
    const int y0 = blockIdx.y * ylen;
    const int y1 = (int)min((int64_t)y0 + ylen, N);
    const int n = y1 - y0 + 2;                                 // rows y0 - 1 .. y1
    const bool down = (blockIdx.y & 1u) != 0;
    // row k of the sweep: y0 - 1 + k upwards, y1 - k downwards (mod N)
    const auto row_off = [&](int k) -> int64_t {
      int64_t y = down ? (int64_t)y1 - k : (int64_t)y0 - 1 + k;
      y = y < 0 ? y + N : (y >= N ? y - N : y);
      return y * N + xs;
    };
    const T c = (T)p.sc_in->c;
    const T dd = p.dt_drift, kk = p.dt_kick, idx2 = p.inv_dx2;
    const T q[3] = {p.q[0], p.q[1], p.q[2]};
    T lf[DL][NF], lw[DL][NF];
    const auto issue = [&](int k, int slot) {
      const int64_t o = row_off(k);
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        lf[slot][i] = __ldg(p.f_in[i] + o);
        lw[slot][i] = __ldg(p.w_in[i] + o);
      }
    };
#pragma unroll
    for (int s = 0; s < DL; ++s)
      if (s < n) issue(s, s);
    T gm[NF], gc[NF], gp[NF], vc[NF], vp[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) gm[i] = gc[i] = gp[i] = vc[i] = vp[i] = T(0);
    int since_flush = 0;
    for (int k0 = 0; k0 < n; k0 += DL) {
#pragma unroll
      for (int s = 0; s < DL; ++s) {
        const int j = k0 + s;
        if (j >= n) break;
#pragma unroll
        for (int i = 0; i < NF; ++i) {
          const T v = fmaT(c, lf[s][i], lw[s][i]);
          gm[i] = gc[i];
          gc[i] = gp[i];
          gp[i] = fmaT(dd, v, lf[s][i]);
          vc[i] = vp[i];
          vp[i] = v;
        }
        if (j + DL < n) issue(j + DL, s);
        if (j < 2) continue;
        // update row j - 1 of the sweep; y + 1 is the next row upwards, the previous one downwards
        T xms[NF], xps[NF];
#pragma unroll
        for (int i = 0; i < NF; ++i) {   // every lane takes part in the shuffles
          xms[i] = __shfl_up_sync(0xffffffffu, gc[i], 1);
          xps[i] = __shfl_down_sync(0xffffffffu, gc[i], 1);
        }
        if (site) {
          T lap[NF];
#pragma unroll
          for (int i = 0; i < NF; ++i) {
            const T g = gc[i];
            const T yp = down ? gm[i] : gp[i], ym = down ? gp[i] : gm[i];
            T acc = T(0);
            acc += (xps[i] + xms[i]) - T(2) * g;
            T df = xps[i] - g;
            g2loc = fmaT(df, df, g2loc);
            acc += (yp + ym) - T(2) * g;
            df = yp - g;
            g2loc = fmaT(df, df, g2loc);
            lap[i] = acc * idx2;
          }
          T dv[NF], vs;
          model_dv<T, NF>(gc, q, dv, vs);
          vloc += vs;
          const int64_t o = row_off(j - 1);
#pragma unroll
          for (int i = 0; i < NF; ++i) {
            __stcs(p.w_out[i] + o, fmaT(kk, lap[i] - dv[i], vc[i]));
            __stcs(p.f_out[i] + o, gc[i]);
          }
        }
        if (++since_flush == 16) {
          g2acc += g2loc;
          vacc += vloc;
          g2loc = T(0);
          vloc = T(0);
          since_flush = 0;
        }
      }
    }
  }
  if (p.update_scalars) finish_step_block(p, (double)g2acc + (double)g2loc, (double)vacc + (double)vloc);
}

template <typename T, int NF>
cudaError_t launch_nf(const StepArgs<T>& a, const LinesPlan& pl, cudaStream_t st) {
  k_step_lines<T, NF, LineDepth<NF>::value><<<dim3(pl.gx, pl.gy), kLineThreads, 0, st>>>(a, pl.nstrips, pl.ylen);
  return cudaGetLastError();
}

template <typename T, int NF>
int blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_lines<T, NF, LineDepth<NF>::value>, kLineThreads,
                                                    0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n < 1 ? 1 : n;
}

}  // namespace

// Grid of the line-sweep kernel: 8 strips of 30 sites per block in x, and the
// row-chunk length of the wave model (plan::wave_chunk_length: chunks of at
// least 8 rows, each costing 5 more for its halo rows and start-up).
LinesPlan lines_plan(int64_t N, int nf, int prec, int sms) {
  LinesPlan pl{};
  pl.nstrips = (int)((N + kStrip - 1) / kStrip);
  pl.gx = (int)((pl.nstrips + kLineWarps - 1) / kLineWarps);
  int per_sm;
  if (prec == CE_F32)
    per_sm = nf == 1 ? blocks_per_sm<float, 1>() : nf == 2 ? blocks_per_sm<float, 2>()
           : nf == 3 ? blocks_per_sm<float, 3>() : blocks_per_sm<float, 4>();
  else
    per_sm = nf == 1 ? blocks_per_sm<double, 1>() : nf == 2 ? blocks_per_sm<double, 2>()
           : nf == 3 ? blocks_per_sm<double, 3>() : blocks_per_sm<double, 4>();
  pl.ylen = plan::wave_chunk_length(N, pl.gx, (int64_t)per_sm * sms, 8, 5.0);   // ce_plan.h
  pl.gy = (int)((N + pl.ylen - 1) / pl.ylen);
  return pl;
}

template <typename T>
cudaError_t launch_step_lines(const StepArgs<T>& a, const LinesPlan& pl, cudaStream_t st) {
  switch (a.nf) {
    case 1: return launch_nf<T, 1>(a, pl, st);
    case 2: return launch_nf<T, 2>(a, pl, st);
    case 3: return launch_nf<T, 3>(a, pl, st);
    default: return launch_nf<T, 4>(a, pl, st);
  }
}
template cudaError_t launch_step_lines<float>(const StepArgs<float>&, const LinesPlan&, cudaStream_t);
template cudaError_t launch_step_lines<double>(const StepArgs<double>&, const LinesPlan&, cudaStream_t);

}  // namespace ce
