// ce_generic.cu -- the generic step (any dimension, any N >= 3): the fused
// one-thread-per-site kernel, its vectorised 1D form, and a two-pass form for
// FP64 in 2D/3D (g written once, then the stencil; FP64 is rate-bound); plus
// the diagnostics pass, the start-up scalar kernel and the host<->device
// conversion kernels of libclusterlat.
//
// The fused step (arXiv:0712.0813 Sec. III staggered leapfrog) per site x and
// field i, with state (f_n, w_n) and v_{n+1/2} = w_n + c_n f_n:
//   v      = w + c f                        expansion kick of the previous step
//   g      = f + dt_drift v                 drift: g = f_{n+1}, also at the 2d neighbours
//   F0     = lap g - dV/df(g)               nearest-neighbour Laplacian (periodic wrap
//                                           by index arithmetic), model force
//   w_out  = v + dt_kick F0,  f_out = g     kick without the (a''/a) f term
// plus block partial sums of sum_d (g(x+e_d) - g(x))^2 and V(g) for the scale
// factor.  f is ping-ponged because neighbours of the old f are still being read
// while the new one is written; the velocity state is ping-ponged for the same
// reason (its neighbours are read to form g there).
#include <atomic>
#include <cstdint>

#include "ce_device.cuh"
#include "ce_internal.h"

namespace ce {

int generic_blocks(int64_t S, int sms) {
  int64_t want = (S + kGenericThreads - 1) / kGenericThreads;
  const int64_t cap = (int64_t)sms * 8;
  return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

int sm_count(int device) {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  if (device < 0 && cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  if (device >= kMaxDevices) device = kMaxDevices - 1;
  int n = cache[device].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n < 1) {
    cudaGetLastError();
    return 1;
  }
  cache[device].store(n, std::memory_order_relaxed);
  return n;
}

// Lattice coordinates along a grid-stride walk s0, s0 + stride, ...: one
// division by N per thread at the start, then additions with carries, so that
// no site pays for a 64-bit division (the row-major index is s = x + N (y + N z)).
template <int DIMS>
struct SiteWalk {
  int64_t x, y, z;      // coordinates of the current site
  int64_t dx, dy, dz;   // the stride in coordinates (each < N, except 1D)
  __device__ __forceinline__ void init(int64_t s0, int64_t stride, int64_t N) {
    y = z = dy = dz = 0;
    if (DIMS == 1) {   // x = s: nothing to wrap inside the walk (s < S = N)
      x = s0;
      dx = stride;
      return;
    }
    x = s0 % N;
    dx = stride % N;
    const int64_t r = s0 / N, dr = stride / N;
    if (DIMS == 2) {
      y = r;
      dy = dr;
    } else {
      y = r % N;
      z = r / N;
      dy = dr % N;
      dz = dr / N;
    }
  }
  // x + dx < 2N and y + dy + 1 < 2N: one conditional subtraction each.  y (2D)
  // and z (3D) leave [0, N) only once the walk has passed the last site.
  __device__ __forceinline__ void advance(int64_t N) {
    x += dx;
    if (DIMS == 1) return;
    int64_t carry = 0;
    if (x >= N) {
      x -= N;
      carry = 1;
    }
    y += dy + carry;
    if (DIMS == 3) {
      carry = 0;
      if (y >= N) {
        y -= N;
        carry = 1;
      }
      z += dz + carry;
    }
  }
};

// The 2 DIMS nearest neighbours of site s at (x, y, z), periodic wrap:
// nb[2d] = s + e_d, nb[2d+1] = s - e_d.
template <int DIMS>
__device__ __forceinline__ void neighbours(int64_t s, const SiteWalk<DIMS>& c, int64_t N, int64_t (&nb)[2 * DIMS]) {
  nb[0] = (c.x == N - 1) ? s - (N - 1) : s + 1;
  nb[1] = (c.x == 0) ? s + (N - 1) : s - 1;
  if (DIMS >= 2) {
    nb[2] = (c.y == N - 1) ? s - (N - 1) * N : s + N;
    nb[3] = (c.y == 0) ? s + (N - 1) * N : s - N;
  }
  if (DIMS >= 3) {
    const int64_t NN = N * N;
    nb[4] = (c.z == N - 1) ? s - (N - 1) * NN : s + NN;
    nb[5] = (c.z == 0) ? s + (N - 1) * NN : s - NN;
  }
}

template <typename T, int NF, int DIMS>
__global__ void __launch_bounds__(kGenericThreads) k_step_generic(const StepArgs<T> p) {
  const T c = (T)p.sc_in->c;
  const T dd = p.dt_drift, kk = p.dt_kick, idx2 = p.inv_dx2;
  const int64_t N = p.N, S = p.S;
  T q[3] = {p.q[0], p.q[1], p.q[2]};
  // sums of the step's global energies: 16 sites in T, then into a second T
  // accumulator, converted to FP64 once per thread.  A flush into FP64 every
  // 16 sites was if-converted into the site loop, which put a float-to-double
  // conversion and an FP64 add per sum and site on GB300's narrow FP64 pipe.
  T g2acc = T(0), vacc = T(0), g2loc = T(0), vloc = T(0);
  int since_flush = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t s0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  SiteWalk<DIMS> at;
  at.init(s0, stride, N);
  for (int64_t s = s0; s < S; s += stride, at.advance(N)) {
    int64_t nb[2 * DIMS];
    neighbours<DIMS>(s, at, N, nb);
    T g[NF], v[NF], lap[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      const T* fi = p.f_in[i];
      const T* wi = p.w_in[i];
      const T f0 = fi[s];
      v[i] = fmaT(c, f0, wi[s]);
      g[i] = fmaT(dd, v[i], f0);
      T acc = T(0);
#pragma unroll
      for (int d = 0; d < DIMS; ++d) {
        const T fp = fi[nb[2 * d]], fm = fi[nb[2 * d + 1]];
        const T gp = fmaT(dd, fmaT(c, fp, wi[nb[2 * d]]), fp);
        const T gm = fmaT(dd, fmaT(c, fm, wi[nb[2 * d + 1]]), fm);
        acc += (gp + gm) - T(2) * g[i];
        const T df = gp - g[i];
        g2loc = fmaT(df, df, g2loc);
      }
      lap[i] = acc * idx2;
    }
    T dv[NF], vs;
    model_dv<T, NF>(g, q, dv, vs);
    vloc += vs;
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      p.w_out[i][s] = fmaT(kk, lap[i] - dv[i], v[i]);
      p.f_out[i][s] = g[i];
    }
    if (++since_flush == 16) {
      g2acc += g2loc;
      vacc += vloc;
      g2loc = T(0);
      vloc = T(0);
      since_flush = 0;
    }
  }
  if (p.update_scalars) finish_step_block(p, (double)g2acc + (double)g2loc, (double)vacc + (double)vloc);
}

// FP64 in 2D and 3D, two passes.  In FP64 the step is bound by GB300's FP64
// rate, and the one-pass kernel forms g = f + dt (w + c f) again for every
// neighbour that reads it (2d + 1 times per site).  Pass 1 writes each site's g
// once, into f_out (which holds g after the step anyway), and v = w + c f into
// w_out (which pass 2 overwrites at the same site, in the same thread); pass 2
// reads the neighbours' g and the site's v from there, sums the 2d neighbours
// once and takes the gradient energy by summation by parts on the periodic lattice,
//   sum_x sum_d (g(x+e_d) - g(x))^2 = -sum_x g(x) raw(x),
//   raw(x) = sum_d (g(x+e_d) + g(x-e_d)) - 2d g(x)
// (exact in exact arithmetic; the cancellation costs ~1e-12 of G in FP64, which
// enters only a'').  About 16 FP64 operations per field and site instead of ~33.
template <int NF>
__global__ void __launch_bounds__(kGenericThreads) k_drift_g(const StepArgs<double> p) {
  const double c = p.sc_in->c, dd = p.dt_drift;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < p.S; s += stride) {
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      const double f = p.f_in[i][s];
      const double v = fma(c, f, p.w_in[i][s]);
      p.w_out[i][s] = v;
      p.f_out[i][s] = fma(dd, v, f);
    }
  }
}

template <int NF, int DIMS>
__global__ void __launch_bounds__(kGenericThreads) k_kick_from_g(const StepArgs<double> p) {
  const double kk = p.dt_kick, idx2 = p.inv_dx2;
  const int64_t N = p.N, S = p.S;
  double q[3] = {p.q[0], p.q[1], p.q[2]};
  double grad2 = 0.0, pot = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t s0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  SiteWalk<DIMS> at;
  at.init(s0, stride, N);
  for (int64_t s = s0; s < S; s += stride, at.advance(N)) {
    int64_t nb[2 * DIMS];
    neighbours<DIMS>(s, at, N, nb);
    double g[NF], lap[NF];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      const double* gi = p.f_out[i];
      g[i] = gi[s];
      double nsum = gi[nb[0]] + gi[nb[1]];
#pragma unroll
      for (int d = 1; d < DIMS; ++d) nsum += gi[nb[2 * d]] + gi[nb[2 * d + 1]];
      const double raw = fma(-2.0 * DIMS, g[i], nsum);
      lap[i] = raw * idx2;
      grad2 = fma(-g[i], raw, grad2);
    }
    double dv[NF], vs;
    model_dv<double, NF>(g, q, dv, vs);
    pot += vs;
#pragma unroll
    for (int i = 0; i < NF; ++i) p.w_out[i][s] = fma(kk, lap[i] - dv[i], p.w_out[i][s]);
  }
  if (p.update_scalars) finish_step_block(p, grad2, pot);
}

// One site s of a 1D lattice with the arithmetic of step1d_group (the sites
// past the last whole 16-byte group of a side that is not a multiple of it).
template <typename T, int NF>
__device__ __forceinline__ void step1d_site(const T* const (&f_in)[4], const T* const (&w_in)[4],
                                            T* const (&f_out)[4], T* const (&w_out)[4], int64_t N, int64_t s,
                                            T c, T dd, T kk, T idx2, const T (&q)[3], T& g2loc, T& vloc) {
  const int64_t sl = (s == 0) ? N - 1 : s - 1, sr = (s == N - 1) ? 0 : s + 1;
  T gs[NF], v[NF], lap[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    const T f = __ldg(f_in[i] + s), fl = __ldg(f_in[i] + sl), fr = __ldg(f_in[i] + sr);
    v[i] = fmaT(c, f, __ldg(w_in[i] + s));
    const T gc = fmaT(dd, v[i], f);
    const T gm = fmaT(dd, fmaT(c, fl, __ldg(w_in[i] + sl)), fl);
    const T gp = fmaT(dd, fmaT(c, fr, __ldg(w_in[i] + sr)), fr);
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
    w_out[i][s] = fmaT(kk, lap[i] - dv[i], v[i]);
    f_out[i][s] = gs[i];
  }
}

// The 1D step for any N: each thread takes groups of VX = 16 / sizeof(T)
// consecutive sites (step1d_group: 16-byte loads and stores, the outer
// neighbours by scalar loads that hit L1, each site's g formed once per field;
// the groups start at site 0, so every 16-byte access is aligned), and the
// grid's last thread the N % VX sites after the last whole group
// (step1d_site).  Per site the arithmetic is that of k_step_generic (same
// operations in the same order), so the fields agree bit for bit; the block
// sums are added in another order.
template <typename T, int NF>
__global__ void __launch_bounds__(kGenericThreads) k_step_1d(const StepArgs<T> p) {
  constexpr int VX = 16 / sizeof(T);
  const T c = (T)p.sc_in->c;
  const T dd = p.dt_drift, kk = p.dt_kick, idx2 = p.inv_dx2;
  const int64_t N = p.N, groups = N / VX;
  const T q[3] = {p.q[0], p.q[1], p.q[2]};
  T g2acc = T(0), vacc = T(0), g2loc = T(0), vloc = T(0);   // two-level sums in T (k_step_generic)
  int since_flush = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < groups; k += stride) {
    step1d_group<T, NF>(p.f_in, p.w_in, p.f_out, p.w_out, N, k, c, dd, kk, idx2, q, g2loc, vloc);
    since_flush += VX;
    if (since_flush >= 16) {
      g2acc += g2loc;
      vacc += vloc;
      g2loc = T(0);
      vloc = T(0);
      since_flush = 0;
    }
  }
  // the N % VX sites after the last whole group: the grid's last thread
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1)
    for (int64_t s = groups * VX; s < N; ++s)
      step1d_site<T, NF>(p.f_in, p.w_in, p.f_out, p.w_out, N, s, c, dd, kk, idx2, q, g2loc, vloc);
  if (p.update_scalars) finish_step_block(p, (double)g2acc + (double)g2loc, (double)vacc + (double)vloc);
}

template <typename T, int NF>
static cudaError_t launch_generic_nf(const StepArgs<T>& a, int blocks, cudaStream_t st) {
  constexpr int VX = 16 / sizeof(T);
  switch (a.dims) {
    case 1: {
      const int64_t want = (a.N / VX + kGenericThreads - 1) / kGenericThreads;
      const int b1 = (int)(want < blocks ? want : blocks);
      k_step_1d<T, NF><<<b1 < 1 ? 1 : b1, kGenericThreads, 0, st>>>(a);
      break;
    }
    case 2: k_step_generic<T, NF, 2><<<blocks, kGenericThreads, 0, st>>>(a); break;
    default: k_step_generic<T, NF, 3><<<blocks, kGenericThreads, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

template <int NF>
static cudaError_t launch_two_pass_nf(const StepArgs<double>& a, int blocks, cudaStream_t st) {
  k_drift_g<NF><<<blocks, kGenericThreads, 0, st>>>(a);
  if (a.dims == 2) k_kick_from_g<NF, 2><<<blocks, kGenericThreads, 0, st>>>(a);
  else k_kick_from_g<NF, 3><<<blocks, kGenericThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step_generic(const StepArgs<T>& a, int blocks, cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    if (a.dims >= 2) {
      switch (a.nf) {
        case 1: return launch_two_pass_nf<1>(a, blocks, st);
        case 2: return launch_two_pass_nf<2>(a, blocks, st);
        case 3: return launch_two_pass_nf<3>(a, blocks, st);
        default: return launch_two_pass_nf<4>(a, blocks, st);
      }
    }
  }
  switch (a.nf) {
    case 1: return launch_generic_nf<T, 1>(a, blocks, st);
    case 2: return launch_generic_nf<T, 2>(a, blocks, st);
    case 3: return launch_generic_nf<T, 3>(a, blocks, st);
    default: return launch_generic_nf<T, 4>(a, blocks, st);
  }
}
template cudaError_t launch_step_generic<float>(const StepArgs<float>&, int, cudaStream_t);
template cudaError_t launch_step_generic<double>(const StepArgs<double>&, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Diagnostics: u(t_n), energies and moments in FP64 (on demand, not per step).
//   v_half = w + c f;  v(t_n) = v_half - dt/2 (lap f - dV/df + s f)
//   a'(t_n) = a'_{n+1/2} - dt/2 a''_n;  u = v(t_n) - (a'(t_n)/a_n) f
// With raw_u (start-up input) u is w itself.

// Per-site quantities in the compute type C: f, u(t_n), the forward-difference
// gradient term sum_d (f(x+e_d) - f(x))^2 and V(f).  The sums (k_diag) use C =
// the storage type, with per-thread partials in C folded into FP64 every 16
// sites as in the step kernels: for FP32 storage the inputs carry 2^-24
// relative rounding already, and FP64 per-site arithmetic (one conversion per
// neighbour load) made the pass bound by GB300's FP64 rate.  The synchronised
// velocity download (k_sync_u_range) uses C = the storage type as well (its
// FP64 form made the download of a 1024^3 FP32 lattice FP64-bound: 0.32 s
// against 0.20 s for the staggered velocity) and converts the result.
template <typename T, typename C, int NF, int DIMS>
__device__ __forceinline__ void site_u(const DiagArgs<T>& p, int64_t s, const SiteWalk<DIMS>& at,
                                       C (&fv)[NF], C (&u)[NF], C (&g2)[NF], C& vsite) {
  int64_t nb[2 * DIMS];
  neighbours<DIMS>(s, at, p.N, nb);
  C lap[NF];
  const C idx2 = (C)p.inv_dx2;
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    const T* fi = p.f[i];
    fv[i] = (C)fi[s];
    C acc = C(0), gg = C(0);
#pragma unroll
    for (int d = 0; d < DIMS; ++d) {
      const C fp = (C)fi[nb[2 * d]], fm = (C)fi[nb[2 * d + 1]];
      acc += (fp + fm) - C(2) * fv[i];
      gg += (fp - fv[i]) * (fp - fv[i]);
    }
    lap[i] = acc * idx2;
    g2[i] = gg;
  }
  C dv[NF];
  C q[3] = {(C)p.q[0], (C)p.q[1], (C)p.q[2]};
  model_dv<C, NF>(fv, q, dv, vsite);
  if (p.raw_u) {
#pragma unroll
    for (int i = 0; i < NF; ++i) u[i] = (C)p.w[i][s];
    return;
  }
  const DevScalars sc = *p.sc;
  const C h = p.expansion ? (C)((sc.ap - 0.5 * p.dt * sc.app) / sc.a) : C(0);
  const C sterm = p.expansion ? (C)sc.s : C(0);
  const C half_dt = (C)(0.5 * p.dt);
  const T cT = (T)sc.c;
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    const T vh = fmaT(cT, p.f[i][s], p.w[i][s]);
    const C vsync = (C)vh - half_dt * (lap[i] - dv[i] + sterm * fv[i]);
    u[i] = vsync - h * fv[i];
  }
}

// partial layout per block: [K_i (NF)][G_i (NF)][V][sum(f_i - f_i(0)) (NF)][sum (f_i - f_i(0))^2 (NF)]
template <typename T, int NF, int DIMS>
__global__ void __launch_bounds__(256) k_diag(const DiagArgs<T> p) {
  constexpr int NV = 4 * NF + 1;
  double acc[NV];
  T part[NV];   // per-thread partials in the storage type, folded into acc every 16 sites
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    acc[k] = 0.0;
    part[k] = T(0);
  }
  T shift[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) shift[i] = p.f[i][0];
  int since_flush = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t s0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  SiteWalk<DIMS> at;
  at.init(s0, stride, p.N);
  for (int64_t s = s0; s < p.S; s += stride, at.advance(p.N)) {
    T fv[NF], u[NF], g2[NF], vs;
    site_u<T, T, NF, DIMS>(p, s, at, fv, u, g2, vs);
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      part[i] += T(0.5) * u[i] * u[i];
      part[NF + i] += g2[i];
      const T df = fv[i] - shift[i];
      part[2 * NF + 1 + i] += df;
      part[3 * NF + 1 + i] += df * df;
    }
    part[2 * NF] += vs;
    if (++since_flush == 16) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        acc[k] += (double)part[k];
        part[k] = T(0);
      }
      since_flush = 0;
    }
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] += (double)part[k];
  __shared__ double red[8][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
    p.partials[(int64_t)blockIdx.x * NV + threadIdx.x] = t;
  }
}

// One block of one warp per quantity: combine the diag partials (lane l takes
// blocks l, l + 32, ..., then a fixed shuffle tree) and derive the outputs.
template <int NF>
__global__ void k_diag_finalize(const double* partials, int blocks, DevAux* aux, int64_t S,
                                double half_inv_dx2, double dt, double kappa2, int expansion,
                                const DevScalars* sc) {
  constexpr int NV = 4 * NF + 1;
  __shared__ double tot[NV];
  const int lane = threadIdx.x & 31;
  for (int k = threadIdx.x >> 5; k < NV; k += blockDim.x >> 5) {
    double t = 0.0;
    for (int b = lane; b < blocks; b += 32) t += partials[(int64_t)b * NV + k];
    t = warp_sum(t);
    if (lane == 0) tot[k] = t;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double* r = aux->result;
  for (int k = 0; k < kResultLen; ++k) r[k] = 0.0;
  const double invS = 1.0 / (double)S;
  double K = 0.0, G = 0.0;
  for (int i = 0; i < NF; ++i) {
    r[R_K + i] = tot[i] * invS;
    r[R_G + i] = tot[NF + i] * half_inv_dx2 * invS;
    K += r[R_K + i];
    G += r[R_G + i];
  }
  r[R_V] = tot[2 * NF] * invS;
  r[R_KTOT] = K;
  r[R_GTOT] = G;
  const double E = K + G + r[R_V];
  r[R_E] = E;
  const DevScalars s = *sc;
  const double ap_t = expansion ? s.ap - 0.5 * dt * s.app : 0.0;
  r[R_A] = expansion ? s.a : 1.0;
  r[R_AP] = ap_t;
  r[R_RESID] = expansion ? fabs(ap_t * ap_t / kappa2 - E) / E : 0.0;
  for (int i = 0; i < NF; ++i) {
    const double m1 = tot[2 * NF + 1 + i] * invS;   // <f - shift>
    const double m2 = tot[3 * NF + 1 + i] * invS;   // <(f - shift)^2>
    r[R_MEAN + i] = m1;                             // k_mean_shift adds the shift back
    r[R_VAR + i] = m2 - m1 * m1;
  }
  if (!isfinite(E)) atomicCAS(&aux->status, CE_OK, CE_ENONFINITE);
}

template <typename T, int NF>
__global__ void k_mean_shift(DevAux* aux, const T* f0, const T* f1, const T* f2, const T* f3) {
  const T* fs[4] = {f0, f1, f2, f3};
  for (int i = 0; i < NF; ++i) aux->result[R_MEAN + i] += (double)fs[i][0];
}

template <typename T, int NF, int DIMS>
__global__ void __launch_bounds__(256) k_sync_u_range(const DiagArgs<T> p) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t k0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  SiteWalk<DIMS> at;
  at.init(p.s0 + k0, stride, p.N);
  for (int64_t k = k0; k < p.count; k += stride, at.advance(p.N)) {
    const int64_t s = p.s0 + k;
    T fv[NF], u[NF], g2[NF], vs;
    site_u<T, T, NF, DIMS>(p, s, at, fv, u, g2, vs);
#pragma unroll
    for (int i = 0; i < NF; ++i) p.u_out[(int64_t)i * p.count + k] = (double)u[i];
  }
}

template <typename T, int NF>
static cudaError_t launch_diag_nf(const DiagArgs<T>& a, int blocks, cudaStream_t st) {
  switch (a.dims) {
    case 1: k_diag<T, NF, 1><<<blocks, 256, 0, st>>>(a); break;
    case 2: k_diag<T, NF, 2><<<blocks, 256, 0, st>>>(a); break;
    default: k_diag<T, NF, 3><<<blocks, 256, 0, st>>>(a); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const double dx2inv = a.inv_dx2;
  k_diag_finalize<NF><<<1, 32 * (4 * NF + 1), 0, st>>>(a.partials, blocks, a.aux, a.S, 0.5 * dx2inv, a.dt, a.kappa2,
                                         a.expansion, a.sc);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_mean_shift<T, NF><<<1, 1, 0, st>>>(a.aux, a.f[0], a.f[NF > 1 ? 1 : 0], a.f[NF > 2 ? 2 : 0],
                                       a.f[NF > 3 ? 3 : 0]);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diag(const DiagArgs<T>& a, int blocks, cudaStream_t st) {
  switch (a.nf) {
    case 1: return launch_diag_nf<T, 1>(a, blocks, st);
    case 2: return launch_diag_nf<T, 2>(a, blocks, st);
    case 3: return launch_diag_nf<T, 3>(a, blocks, st);
    default: return launch_diag_nf<T, 4>(a, blocks, st);
  }
}
template cudaError_t launch_diag<float>(const DiagArgs<float>&, int, cudaStream_t);
template cudaError_t launch_diag<double>(const DiagArgs<double>&, int, cudaStream_t);

template <typename T, int NF>
static cudaError_t launch_sync_nf(const DiagArgs<T>& a, cudaStream_t st) {
  const int64_t want = (a.count + 255) / 256, cap = (int64_t)sm_count(-1) * 16;
  int blocks = (int)(want < cap ? want : cap);
  if (blocks < 1) blocks = 1;
  switch (a.dims) {
    case 1: k_sync_u_range<T, NF, 1><<<blocks, 256, 0, st>>>(a); break;
    case 2: k_sync_u_range<T, NF, 2><<<blocks, 256, 0, st>>>(a); break;
    default: k_sync_u_range<T, NF, 3><<<blocks, 256, 0, st>>>(a); break;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sync_u_range(const DiagArgs<T>& a, cudaStream_t st) {
  switch (a.nf) {
    case 1: return launch_sync_nf<T, 1>(a, st);
    case 2: return launch_sync_nf<T, 2>(a, st);
    case 3: return launch_sync_nf<T, 3>(a, st);
    default: return launch_sync_nf<T, 4>(a, st);
  }
}
template cudaError_t launch_sync_u_range<float>(const DiagArgs<float>&, cudaStream_t);
template cudaError_t launch_sync_u_range<double>(const DiagArgs<double>&, cudaStream_t);

// ---------------------------------------------------------------------------
// Start-up scalars (reading c-6), one thread, after a raw-u diagnostics pass
// over (f(0), u(0)):  a = 1, a'(0) = sqrt(kappa2 (K + G + V)),
//   a''(0) = (-a'(0)^2 + kappa2 (2G + 3V)) / a.
// slot[cur]   feeds the half-kick launch: c = a'(0)/a turns u into f'(0).
// slot[cur^1] is the state after it: a'(dt/2) = a'(0) + dt/2 a''(0) and
//             c = dt/2 a''(0)/a, the expansion half of the half kick.
__global__ void k_init_scalars(DevAux* aux, int cur, int expansion, double dt, double kappa2) {
  const double* r = aux->result;
  const double K = r[R_KTOT], G = r[R_GTOT], V = r[R_V];
  double ap0 = 0.0, app0 = 0.0;
  const double a = 1.0;
  if (expansion) {
    const double rho = K + G + V;
    if (!(rho >= 0.0) || !isfinite(rho)) atomicCAS(&aux->status, CE_OK, CE_ENONFINITE);
    ap0 = sqrt(kappa2 * rho);
    app0 = (-ap0 * ap0 + kappa2 * (2.0 * G + 3.0 * V)) / a;
  }
  DevScalars s0;
  s0.a = a; s0.ap = ap0; s0.app = 0.0; s0.s = 0.0; s0.c = ap0 / a; s0.G = G; s0.V = V; s0.pad = 0.0;
  DevScalars s1;
  s1.a = a;
  s1.ap = ap0 + 0.5 * dt * app0;
  s1.app = app0;
  s1.s = app0 / a;
  s1.c = 0.5 * dt * s1.s;
  s1.G = G; s1.V = V; s1.pad = 0.0;
  aux->slot[cur] = s0;
  aux->slot[cur ^ 1] = s1;
}

cudaError_t launch_init_scalars(DevAux* aux, int cur, int expansion, double dt, double kappa2,
                                cudaStream_t st) {
  k_init_scalars<<<1, 1, 0, st>>>(aux, cur, expansion, dt, kappa2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Conversions between the caller's float64 host layout (staged in HBM) and the
// storage type.

template <typename T>
__global__ void k_from_f64(const double* __restrict__ src, T* __restrict__ dst, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) dst[k] = (T)src[k];
}

template <typename T>
__global__ void k_to_f64(const T* __restrict__ src, double* __restrict__ dst, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) dst[k] = (double)src[k];
}

// f'(t+dt/2) = w + c f, rounded in T exactly as the step kernel forms it.
template <typename T>
__global__ void k_vhalf_to_f64(const T* __restrict__ f, const T* __restrict__ w, const DevScalars* sc,
                               double* __restrict__ dst, int64_t n) {
  const T c = (T)sc->c;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
    dst[k] = (double)fmaT(c, f[k], w[k]);
}

static int conv_blocks(int64_t n) {
  const int64_t want = (n + 255) / 256, cap = (int64_t)sm_count(-1) * 16;
  return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

template <typename T>
cudaError_t launch_from_f64(const double* src, T* dst, int64_t n, cudaStream_t st) {
  k_from_f64<T><<<conv_blocks(n), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_to_f64(const T* src, double* dst, int64_t n, cudaStream_t st) {
  k_to_f64<T><<<conv_blocks(n), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_vhalf_to_f64(const T* f, const T* w, const DevScalars* sc, double* dst, int64_t n,
                                cudaStream_t st) {
  k_vhalf_to_f64<T><<<conv_blocks(n), 256, 0, st>>>(f, w, sc, dst, n);
  return cudaGetLastError();
}
template cudaError_t launch_from_f64<float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_from_f64<double>(const double*, double*, int64_t, cudaStream_t);
template cudaError_t launch_to_f64<float>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_to_f64<double>(const double*, double*, int64_t, cudaStream_t);
template cudaError_t launch_vhalf_to_f64<float>(const float*, const float*, const DevScalars*, double*,
                                                int64_t, cudaStream_t);
template cudaError_t launch_vhalf_to_f64<double>(const double*, const double*, const DevScalars*,
                                                 double*, int64_t, cudaStream_t);

}  // namespace ce
