// ce_device.cuh -- device-side building blocks shared by the step kernels:
// the model (potential and its derivatives), the block reduction of the
// global sums, and the scale-factor update done by the last block of a step.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ce_internal.h"

namespace ce {

__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }

// Model V = phi^4/4 + sum_i (q_i/2) phi^2 chi_i^2 (program units) at one site:
// dV/df for each field and V itself.  g[0] = phi, g[i>0] = chi_i.
template <typename T, int NF>
__device__ __forceinline__ void model_dv(const T (&g)[NF], const T (&q)[3], T (&dv)[NF], T& vsite) {
  const T phi = g[0];
  const T phi2 = phi * phi;
  T cpl = T(0);  // sum_i q_i chi_i^2
#pragma unroll
  for (int i = 1; i < NF; ++i) cpl = fmaT(q[i - 1] * g[i], g[i], cpl);
  dv[0] = phi * fmaT(phi, phi, cpl);
#pragma unroll
  for (int i = 1; i < NF; ++i) dv[i] = q[i - 1] * phi2 * g[i];
  vsite = phi2 * fmaT(T(0.25), phi2, T(0.5) * cpl);
}

// 16 bytes of consecutive sites: VX = 16 / sizeof(T) values, one vector access
// (read-only path for loads, streaming stores).
template <typename T, int VX>
__device__ __forceinline__ void ldg16v(const T* p, T (&o)[VX]) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = v.x; o[1] = v.y;
  }
}
template <typename T, int VX>
__device__ __forceinline__ void stcs16v(T* p, const T (&o)[VX]) {
  if constexpr (sizeof(T) == 4) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(o[0], o[1], o[2], o[3]));
  } else {
    __stcs(reinterpret_cast<double2*>(p), make_double2(o[0], o[1]));
  }
}

// One 16-byte group of the 1D step: VX = 16 / sizeof(T) consecutive sites
// starting at site s = k VX of a periodic 1D lattice of N sites (N a multiple
// of VX), all fields.  16-byte loads of the group's f and w, scalar loads of the
// two outer neighbours (the neighbouring groups' vectors already brought them
// into L1), each site's g = f + dd (w + c f) formed once per field, then
// w_out = v + kk (lap g - dV/df(g)) and f_out = g with 16-byte streaming stores.
// The per-site operations and their order are those of the generic kernel, so
// every 1D kernel built on this gives the same fields bit for bit.  Adds the
// group's sum of (g(x+1) - g(x))^2 and of V(g) to g2loc and vloc.
template <typename T, int NF>
__device__ __forceinline__ void step1d_group(const T* const (&f_in)[4], const T* const (&w_in)[4],
                                             T* const (&f_out)[4], T* const (&w_out)[4], int64_t N, int64_t k,
                                             T c, T dd, T kk, T idx2, const T (&q)[3], T& g2loc, T& vloc) {
  constexpr int VX = 16 / sizeof(T);
  const int64_t s = k * VX;
  const int64_t sl = (k == 0) ? N - 1 : s - 1;             // left neighbour of the first site
  const int64_t sr = (s + VX == N) ? 0 : s + VX;           // right neighbour of the last site
  T g[NF][VX + 2], v[NF][VX];   // g[i][1 + j] at site s + j; [0] and [VX + 1] the outer neighbours
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    T f[VX], w[VX];
    ldg16v<T, VX>(f_in[i] + s, f);
    ldg16v<T, VX>(w_in[i] + s, w);
#pragma unroll
    for (int j = 0; j < VX; ++j) {
      v[i][j] = fmaT(c, f[j], w[j]);
      g[i][j + 1] = fmaT(dd, v[i][j], f[j]);
    }
    const T fl = __ldg(f_in[i] + sl), wl = __ldg(w_in[i] + sl);
    const T fr = __ldg(f_in[i] + sr), wr = __ldg(w_in[i] + sr);
    g[i][0] = fmaT(dd, fmaT(c, fl, wl), fl);
    g[i][VX + 1] = fmaT(dd, fmaT(c, fr, wr), fr);
  }
  T wo[NF][VX], fo[NF][VX];
#pragma unroll
  for (int j = 0; j < VX; ++j) {
    T gs[NF], lap[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      const T gc = g[i][j + 1], gp = g[i][j + 2], gm = g[i][j];
      T acc = T(0);
      acc += (gp + gm) - T(2) * gc;
      const T df = gp - gc;
      g2loc = fmaT(df, df, g2loc);
      lap[i] = acc * idx2;
      gs[i] = gc;
    }
    T dv[NF], vs;
    model_dv<T, NF>(gs, q, dv, vs);
    vloc += vs;
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      wo[i][j] = fmaT(kk, lap[i] - dv[i], v[i][j]);
      fo[i][j] = gs[i];
    }
  }
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    stcs16v<T, VX>(w_out[i] + s, wo[i]);
    stcs16v<T, VX>(f_out[i] + s, fo[i]);
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int64_t linear_block_id() {
  return (int64_t)blockIdx.x + (int64_t)gridDim.x * ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
}

__device__ __forceinline__ int64_t grid_blocks() {
  return (int64_t)gridDim.x * gridDim.y * gridDim.z;
}

// Fixed-order block sum of two values; the result is valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) { sa[warp] = a; sb[warp] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < nwarps; ++w) { x += sa[w]; y += sb[w]; }
    a = x;
    b = y;
  }
  __syncthreads();
}

// Block sum of two per-thread values of the storage type T: a fixed tree of
// shuffles inside each warp in T, then the warps' sums added in FP64, in warp
// order, by thread 0.  For T = float this keeps the FP64 work of a block at
// two additions per warp (GB300's FP64 pipe is narrow: a warp-wide FP64
// instruction occupies it for 16 cycles); the tree over 32 values adds at most
// ~5 rounding steps of 2^-24 to each warp's sum.  Result valid in thread 0.
template <typename T>
__device__ __forceinline__ void block_sum2_t(T a, T b, double& oa, double& ob) {
  __shared__ double sa[32], sb[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    sa[warp] = (double)a;
    sb[warp] = (double)b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < nwarps; ++w) {
      x += sa[w];
      y += sb[w];
    }
    oa = x;
    ob = y;
  }
  __syncthreads();
}

// Scale-factor update of reading c-4, done once per step by one thread:
//   a_{n+1} = a_n + dt a'_{n+1/2}
//   Q = kappa2 (2 G + 3 V) / a_{n+1},  C = 2 a'_{n+1/2} + dt Q
//   u = a'_{n+3/2} + a'_{n+1/2} = 2 C / (1 + sqrt(1 + dt C / a_{n+1}))
// (closed form of the implicit midpoint a'_new - a'_old = dt (-(u/2)^2/a + Q)),
//   a''_{n+1} = (u - 2 a'_{n+1/2}) / dt,  a'_{n+3/2} = u - a'_{n+1/2}.
__device__ __forceinline__ void scale_factor_update(const DevScalars& in, DevScalars& out, double G,
                                                    double V, double dt, double kappa2, int* status) {
  const double a = in.a + dt * in.ap;
  const double Q = kappa2 * (2.0 * G + 3.0 * V) / a;
  const double C = 2.0 * in.ap + dt * Q;
  const double disc = 1.0 + dt * C / a;
  if (!(disc >= 0.0) || !isfinite(G) || !isfinite(V)) atomicCAS(status, CE_OK, CE_ENONFINITE);
  const double u = 2.0 * C / (1.0 + sqrt(disc));
  const double app = (u - 2.0 * in.ap) / dt;
  out.a = a;
  out.ap = u - in.ap;
  out.app = app;
  out.s = app / a;
  out.c = dt * out.s;
  out.G = G;
  out.V = V;
  out.pad = 0.0;
}

// End of a step launch: reduce this block's partial sums of
//   sum (f(x+e_d) - f(x))^2   and   sum V(f(x))
// in a fixed order, publish them, and let the last block to finish combine all
// blocks' partials (fixed order over block index) and advance a, a', a''.
// No block ever waits for another: the last arriving block does the work.
template <typename T>
__device__ __forceinline__ void finish_step_block(const StepArgs<T>& p, double grad2, double pot) {
  __shared__ int am_last;
  block_sum2(grad2, pot);
  const int64_t nb = grid_blocks();
  if (threadIdx.x == 0) {
    const int64_t b = linear_block_id();
    p.partials[2 * b] = grad2;
    p.partials[2 * b + 1] = pot;
    __threadfence();
    const unsigned int prev = atomicAdd(p.counter, 1u);
    am_last = (prev == (unsigned int)(nb - 1));
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  double g = 0.0, v = 0.0;
  for (int64_t j = threadIdx.x; j < nb; j += blockDim.x) {
    g += __ldcg(p.partials + 2 * j);
    v += __ldcg(p.partials + 2 * j + 1);
  }
  block_sum2(g, v);
  if (threadIdx.x == 0) {
    DevScalars out;
    scale_factor_update(*p.sc_in, out, g * p.half_inv_dx2 * p.inv_S, v * p.inv_S, p.dt, p.kappa2,
                        p.status);
    *p.sc_out = out;
    *p.counter = 0u;
  }
}

}  // namespace ce
