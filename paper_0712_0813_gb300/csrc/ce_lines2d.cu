// ce_lines2d.cu -- the 2D step for any side N: each warp sweeps a 32-site
// strip of x along a chunk of rows y, with plain coalesced loads (no
// alignment needed, so odd sides work), y-neighbours carried in registers and
// x-neighbours exchanged by warp shuffles: no shared memory, no block barrier
// in the sweep.
//
// Per site the arithmetic is the generic kernel's (arXiv:0712.0813 Sec. III
// staggered leapfrog, fused: v = w + c f, g = f + dt v, lap g from the 2d
// nearest neighbours in the order x, y, w_out = v + dt (lap g - dV/df(g)),
// f_out = g), so the fields agree with k_step_generic bit for bit; only the
// global sums are added in another order.
//
// Warp w of block b owns the strip x0 = 32 (8 b.x + w) .. x0 + nx - 1 (nx <= 32)
// and the rows y0 .. y1 - 1 of chunk b.y; it forms g on the rows y0 - 1 .. y1
// (mod N).  The strip's x-halo: lane 0 also forms g at x0 - 1; the site
// x0 + nx (mod N) is formed by lane nx as if it were its own when nx < 32 (the
// shuffle then brings it to lane nx - 1), and by lane 31 beside its own
// otherwise.  Each thread keeps the loads of the next two rows in
// flight (registers), so a warp has 2 x 4 NF values of 4 or 8 bytes per lane
// outstanding.
#include <cstdint>

#include "ce_device.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

constexpr int kLineWarps = 8;
constexpr int kLineThreads = 32 * kLineWarps;

template <typename T, int NF>
__global__ void __launch_bounds__(kLineThreads) k_step_lines(const StepArgs<T> p, int ylen) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t N = p.N;
  const int64_t x0 = ((int64_t)blockIdx.x * kLineWarps + warp) * 32;
  const int y0 = blockIdx.y * ylen;
  const int y1 = (int)min((int64_t)y0 + ylen, N);
  T g2acc = T(0), vacc = T(0), g2loc = T(0), vloc = T(0);   // two-level sums (see k_step_generic)
  if (x0 < N) {
    const int nx = (int)min((int64_t)32, N - x0);
    const int64_t xl = x0 == 0 ? N - 1 : x0 - 1, xr = x0 + nx == N ? 0 : x0 + nx;
    const bool site = lane < nx;                              // updates a site
    const bool act = lane <= nx && lane < 32;                 // forms a g: the site, or lane nx the right halo
    const bool hl = lane == 0, hr = nx == 32 && lane == 31;   // halo g beside the own one
    const int64_t xs = lane < nx ? x0 + lane : xr;
    const T c = (T)p.sc_in->c;
    const T dd = p.dt_drift, kk = p.dt_kick, idx2 = p.inv_dx2;
    const T q[3] = {p.q[0], p.q[1], p.q[2]};
    const int n = y1 - y0 + 2;                                // staged rows y0 - 1 .. y1
    int64_t yrow = y0 == 0 ? N - 1 : y0 - 1;                  // row of the next load
    // loads in flight: A = the next row, B = the one after it
    T fa[NF], wa[NF], fha[NF], wha[NF], fb[NF], wb[NF], fhb[NF], whb[NF];
    const auto fetch = [&](T (&f)[NF], T (&w)[NF], T (&fh)[NF], T (&wh)[NF]) {
      const int64_t base = yrow * N;
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        if (act) {
          f[i] = __ldg(p.f_in[i] + base + xs);
          w[i] = __ldg(p.w_in[i] + base + xs);
        }
        if (hl || hr) {
          const int64_t hx = hl ? xl : xr;
          fh[i] = __ldg(p.f_in[i] + base + hx);
          wh[i] = __ldg(p.w_in[i] + base + hx);
        }
      }
      yrow = yrow == N - 1 ? 0 : yrow + 1;
    };
    T gm[NF], gc[NF], gp[NF], vc[NF], vn[NF], hc[NF], hp[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) gm[i] = gc[i] = gp[i] = vc[i] = vn[i] = hc[i] = hp[i] = T(0);
    int since_flush = 0;
    int64_t upd = (int64_t)y0 * N + xs;                       // output offset of the next updated row
    // staged row j (loads in f, w, fh, wh): form its g into gp (own site) and
    // hp (halo site); then (j >= 2) update row j - 1
    const auto stage = [&](int j, const T (&f)[NF], const T (&w)[NF], const T (&fh)[NF], const T (&wh)[NF]) {
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        gm[i] = gc[i];
        gc[i] = gp[i];
        vc[i] = vn[i];
        hc[i] = hp[i];
        if (act) {
          vn[i] = fmaT(c, f[i], w[i]);
          gp[i] = fmaT(dd, vn[i], f[i]);
        }
        if (hl || hr) hp[i] = fmaT(dd, fmaT(c, fh[i], wh[i]), fh[i]);
      }
      if (j < 2) return;
      T xms[NF], xps[NF];
#pragma unroll
      for (int i = 0; i < NF; ++i) {   // every lane takes part in the shuffles
        xms[i] = __shfl_up_sync(0xffffffffu, gc[i], 1);
        xps[i] = __shfl_down_sync(0xffffffffu, gc[i], 1);
      }
      if (!site) return;
      T lap[NF];
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        const T g = gc[i];
        const T xm = hl ? hc[i] : xms[i];
        const T xp = hr ? hc[i] : xps[i];
        T acc = T(0);
        acc += (xp + xm) - T(2) * g;
        T df = xp - g;
        g2loc = fmaT(df, df, g2loc);
        acc += (gp[i] + gm[i]) - T(2) * g;
        df = gp[i] - g;
        g2loc = fmaT(df, df, g2loc);
        lap[i] = acc * idx2;
      }
      T dv[NF], vs;
      model_dv<T, NF>(gc, q, dv, vs);
      vloc += vs;
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        __stcs(p.w_out[i] + upd, fmaT(kk, lap[i] - dv[i], vc[i]));
        __stcs(p.f_out[i] + upd, gc[i]);
      }
      upd += N;   // the chunk's rows y0 .. y1 - 1 do not wrap
      if (++since_flush == 16) {
        g2acc += g2loc;
        vacc += vloc;
        g2loc = T(0);
        vloc = T(0);
        since_flush = 0;
      }
    };
    fetch(fa, wa, fha, wha);
    if (n > 1) fetch(fb, wb, fhb, whb);
    for (int j = 0; j < n; j += 2) {
      T f[NF], w[NF], fh[NF], wh[NF];
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        f[i] = fa[i];
        w[i] = wa[i];
        fh[i] = fha[i];
        wh[i] = wha[i];
      }
      if (j + 2 < n) fetch(fa, wa, fha, wha);
      stage(j, f, w, fh, wh);
      if (j + 1 < n) {
#pragma unroll
        for (int i = 0; i < NF; ++i) {
          f[i] = fb[i];
          w[i] = wb[i];
          fh[i] = fhb[i];
          wh[i] = whb[i];
        }
        if (j + 3 < n) fetch(fb, wb, fhb, whb);
        stage(j + 1, f, w, fh, wh);
      }
    }
  }
  if (p.update_scalars) finish_step_block(p, (double)g2acc + (double)g2loc, (double)vacc + (double)vloc);
}

template <typename T, int NF>
cudaError_t launch_nf(const StepArgs<T>& a, const LinesPlan& pl, cudaStream_t st) {
  k_step_lines<T, NF><<<dim3(pl.gx, pl.gy), kLineThreads, 0, st>>>(a, pl.ylen);
  return cudaGetLastError();
}

template <typename T, int NF>
int blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_step_lines<T, NF>, kLineThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n < 1 ? 1 : n;
}

}  // namespace

// Grid of the line-sweep kernel: 8 strips of 32 sites per block in x, y split
// into chunks so that about two waves of resident blocks are busy, with chunks
// of at least 16 rows (each chunk forms 2 halo rows besides its own).
LinesPlan lines_plan(int64_t N, int nf, int prec, int sms) {
  LinesPlan pl{};
  const int64_t strips = (N + 31) / 32;
  pl.gx = (int)((strips + kLineWarps - 1) / kLineWarps);
  int per_sm;
  if (prec == CE_F32)
    per_sm = nf == 1 ? blocks_per_sm<float, 1>() : nf == 2 ? blocks_per_sm<float, 2>()
           : nf == 3 ? blocks_per_sm<float, 3>() : blocks_per_sm<float, 4>();
  else
    per_sm = nf == 1 ? blocks_per_sm<double, 1>() : nf == 2 ? blocks_per_sm<double, 2>()
           : nf == 3 ? blocks_per_sm<double, 3>() : blocks_per_sm<double, 4>();
  const int64_t want = std::max<int64_t>(1, (2LL * per_sm * sms + pl.gx - 1) / pl.gx);
  const int64_t gy = std::max<int64_t>(1, std::min<int64_t>(want, N / 16));
  pl.ylen = (int)((N + gy - 1) / gy);
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
