// ce_sweep3d.cu -- the 3D z-sweep fused leapfrog step for sm_103a.
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
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "ce_device.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

constexpr int kTY = 8;
constexpr int kStages = 4;
constexpr uint32_t kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, P;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
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
__global__ void __launch_bounds__(32 * TY) k_step_sweep(const StepArgs<T> p,
                                                        const __grid_constant__ SweepMaps maps) {
  constexpr int VX = 16 / sizeof(T);
  constexpr int TX = 32 * VX;
  constexpr int PLANE = (TY + 2) * TX;  // elements of one array in one stage
  constexpr uint32_t kPlaneBytes = 2u * NF * PLANE * sizeof(T);
  extern __shared__ __align__(128) unsigned char smem_dyn[];
  // TMA destinations are kept 128-byte aligned whatever the static smem layout.
  unsigned char* smem_raw = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 127) & ~static_cast<uintptr_t>(127));
  T* stage = reinterpret_cast<T*>(smem_raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)NST * NF * 2 * PLANE * sizeof(T));

  const int lane = threadIdx.x & 31;
  const int r = threadIdx.x >> 5;  // row of the tile this warp owns
  const int N = (int)p.N;
  const int64_t NN = (int64_t)N * N;
  const int x0 = blockIdx.x * TX;
  const int y0 = blockIdx.y * TY;
  const int z0 = (int)(((int64_t)blockIdx.z * N) / gridDim.z);
  const int z1 = (int)(((int64_t)(blockIdx.z + 1) * N) / gridDim.z);
  const int nplanes = z1 - z0 + 2;  // planes z0-1 .. z1

  const T c = (T)p.sc_in->c;
  const T dd = p.dt_drift, kk = p.dt_kick, idx2 = p.inv_dx2;
  T q[3] = {p.q[0], p.q[1], p.q[2]};

  auto sbuf = [&](int slot, int i, int a) -> T* {
    return stage + ((size_t)(slot * NF + i) * 2 + a) * PLANE;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // Plane pidx (z = z0 - 1 + pidx, wrapped) of every field's f and w into ring slot pidx % NST.
  auto issue = [&](int pidx) {
    const int slot = pidx % NST;
    int zz = z0 - 1 + pidx;
    zz = zz < 0 ? zz + N : (zz >= N ? zz - N : zz);
    mbar_expect_tx(&bars[slot], kPlaneBytes);
#pragma unroll
    for (int i = 0; i < NF; ++i) {
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        T* dst = sbuf(slot, i, a);
        if (y0 == 0) {
          tma_load_3d(dst + TX, &maps.m[i][a][1], x0, 0, zz, &bars[slot]);
          tma_load_3d(dst, &maps.m[i][a][2], x0, N - 1, zz, &bars[slot]);
        } else if (y0 + TY == N) {
          tma_load_3d(dst, &maps.m[i][a][1], x0, y0 - 1, zz, &bars[slot]);
          tma_load_3d(dst + (TY + 1) * TX, &maps.m[i][a][2], x0, 0, zz, &bars[slot]);
        } else {
          tma_load_3d(dst, &maps.m[i][a][0], x0, y0 - 1, zz, &bars[slot]);
        }
      }
    }
  };

  bool ok = true;
  int waited = 0;  // planes [0, waited) have landed (as seen by this thread)
  auto wait_plane = [&](int pidx) {
    const int slot = pidx % NST;
    const uint32_t parity = (uint32_t)(pidx / NST) & 1u;
    uint32_t it = 0;
    while (!mbar_try_wait(&bars[slot], parity)) {
      if (++it >= kSpinLimit) {
        ok = false;
        return;
      }
    }
    waited = pidx + 1;
  };

  if (threadIdx.x == 0) {
    const int np = nplanes < NST ? nplanes : NST;
    for (int k = 0; k < np; ++k) issue(k);
  }

  // Row-end halo in x: lane 0 needs x0 - 1, lane 31 needs x0 + TX (wrapped).
  const bool hlane = (lane == 0) || (lane == 31);
  const int hx = (lane == 0) ? (x0 == 0 ? N - 1 : x0 - 1) : (x0 + TX == N ? 0 : x0 + TX);
  const int64_t hrow = (int64_t)(y0 + r) * N + hx;
  T hf0[NF], hw0[NF], hf1[NF], hw1[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    hf0[i] = hw0[i] = hf1[i] = hw1[i] = T(0);
    if (hlane) {
      hf0[i] = __ldg(p.f_in[i] + (int64_t)z0 * NN + hrow);
      hw0[i] = __ldg(p.w_in[i] + (int64_t)z0 * NN + hrow);
      if (z0 + 1 < z1) {
        hf1[i] = __ldg(p.f_in[i] + (int64_t)(z0 + 1) * NN + hrow);
        hw1[i] = __ldg(p.w_in[i] + (int64_t)(z0 + 1) * NN + hrow);
      }
    }
  }

  const int col = lane * VX;  // first column of this thread in the tile
  T gp[NF][VX], gc[NF][VX], vc[NF][VX];
  // prologue: plane z0 - 1 (g only) and plane z0 (g and v) at the own sites
  wait_plane(0);
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    T f[VX], w[VX];
    lds16<T, VX>(sbuf(0, i, 0) + (r + 1) * TX + col, f);
    lds16<T, VX>(sbuf(0, i, 1) + (r + 1) * TX + col, w);
#pragma unroll
    for (int j = 0; j < VX; ++j) gp[i][j] = fmaT(dd, fmaT(c, f[j], w[j]), f[j]);
  }
  wait_plane(1);
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
  bool timed_out = __syncthreads_or(!ok);
  if (!timed_out && threadIdx.x == 0 && NST < nplanes) issue(NST);

  double grad2 = 0.0, pot = 0.0;
  T g2loc = T(0), vloc = T(0);
  int issued = (NST < nplanes) ? NST + 1 : nplanes;  // planes handed to TMA so far

  for (int z = z0; z < z1 && !timed_out; ++z) {
    const int pc = z - z0 + 1;  // plane index of z
    const int pn = pc + 1;      // plane index of z + 1 (always <= nplanes - 1)
    wait_plane(pn);
    const int sc_cur = pc % NST, sc_nxt = pn % NST;

    T gn[NF][VX], vn[NF][VX], lap[NF][VX];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      // next plane, own sites
      {
        T f[VX], w[VX];
        lds16<T, VX>(sbuf(sc_nxt, i, 0) + (r + 1) * TX + col, f);
        lds16<T, VX>(sbuf(sc_nxt, i, 1) + (r + 1) * TX + col, w);
#pragma unroll
        for (int j = 0; j < VX; ++j) {
          vn[i][j] = fmaT(c, f[j], w[j]);
          gn[i][j] = fmaT(dd, vn[i][j], f[j]);
        }
      }
      // y neighbours in the current plane
      T ym[VX], yp[VX];
      {
        T f[VX], w[VX];
        lds16<T, VX>(sbuf(sc_cur, i, 0) + r * TX + col, f);
        lds16<T, VX>(sbuf(sc_cur, i, 1) + r * TX + col, w);
#pragma unroll
        for (int j = 0; j < VX; ++j) ym[j] = fmaT(dd, fmaT(c, f[j], w[j]), f[j]);
        lds16<T, VX>(sbuf(sc_cur, i, 0) + (r + 2) * TX + col, f);
        lds16<T, VX>(sbuf(sc_cur, i, 1) + (r + 2) * TX + col, w);
#pragma unroll
        for (int j = 0; j < VX; ++j) yp[j] = fmaT(dd, fmaT(c, f[j], w[j]), f[j]);
      }
      // x neighbours: adjacent lanes, halo at the row ends
      const T gh = fmaT(dd, fmaT(c, hf0[i], hw0[i]), hf0[i]);
      T gl = __shfl_up_sync(0xffffffffu, gc[i][VX - 1], 1);
      T gr = __shfl_down_sync(0xffffffffu, gc[i][0], 1);
      if (lane == 0) gl = gh;
      if (lane == 31) gr = gh;
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        const T g = gc[i][j];
        const T xm = (j == 0) ? gl : gc[i][j - 1];
        const T xp = (j == VX - 1) ? gr : gc[i][j + 1];
        T acc = T(0);
        acc += (xp + xm) - T(2) * g;
        acc += (yp[j] + ym[j]) - T(2) * g;
        acc += (gn[i][j] + gp[i][j]) - T(2) * g;
        lap[i][j] = acc * idx2;
        const T dx = xp - g, dy = yp[j] - g, dz = gn[i][j] - g;
        g2loc = fmaT(dx, dx, g2loc);
        g2loc = fmaT(dy, dy, g2loc);
        g2loc = fmaT(dz, dz, g2loc);
      }
    }
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
    if (((z - z0) & 7) == 7) {
      grad2 += (double)g2loc;
      pot += (double)vloc;
      g2loc = T(0);
      vloc = T(0);
    }
    // rotate the register window and the x-halo ring
#pragma unroll
    for (int i = 0; i < NF; ++i) {
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        gp[i][j] = gc[i][j];
        gc[i][j] = gn[i][j];
        vc[i][j] = vn[i][j];
      }
      hf0[i] = hf1[i];
      hw0[i] = hw1[i];
      if (hlane && z + 2 < z1) {
        hf1[i] = __ldg(p.f_in[i] + (int64_t)(z + 2) * NN + hrow);
        hw1[i] = __ldg(p.w_in[i] + (int64_t)(z + 2) * NN + hrow);
      }
    }
    timed_out = __syncthreads_or(!ok);
    if (!timed_out && threadIdx.x == 0 && pc + NST < nplanes) {
      issue(pc + NST);
      issued = pc + NST + 1;
    }
  }

  if (timed_out) {
    // Latch the error, then give the copies this CTA still has in flight a
    // bounded chance to land before shared memory is released.
    if (threadIdx.x == 0) {
      atomicCAS(p.status, CE_OK, CE_ETIMEOUT);
      for (int k = waited; k < issued; ++k) {
        const int slot = k % NST;
        const uint32_t parity = (uint32_t)(k / NST) & 1u;
        uint32_t it = 0;
        while (!mbar_try_wait(&bars[slot], parity) && ++it < kSpinLimit) {
        }
      }
    }
    __syncthreads();
    grad2 = 0.0;
    pot = 0.0;
    g2loc = T(0);
    vloc = T(0);
  }
  if (p.update_scalars) {
    grad2 += (double)g2loc;
    pot += (double)vloc;
    finish_step_block(p, grad2, pot);
  }
}

template <typename T, int NF>
constexpr auto sweep_kernel() {
  return &k_step_sweep<T, NF, kTY, kStages>;
}

template <typename T>
size_t sweep_smem_bytes(int nf) {
  constexpr int VX = 16 / sizeof(T);
  constexpr int TX = 32 * VX;
  return (size_t)kStages * nf * 2 * (kTY + 2) * TX * sizeof(T) + kStages * sizeof(uint64_t) + 128;
}

template <typename T>
const void* sweep_kernel_ptr(int nf) {
  switch (nf) {
    case 1: return (const void*)sweep_kernel<T, 1>();
    case 2: return (const void*)sweep_kernel<T, 2>();
    case 3: return (const void*)sweep_kernel<T, 3>();
    default: return (const void*)sweep_kernel<T, 4>();
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encoder() {
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

}  // namespace

bool sweep_supported(int dims, int64_t N, int nf, int prec) {
  const int tx = prec == CE_F32 ? 128 : 64;
  if (dims != 3 || nf < 1 || nf > 4) return false;
  if (N % tx != 0 || N % kTY != 0 || N < 2 * kTY || N > (1 << 20)) return false;
  const size_t smem = prec == CE_F32 ? sweep_smem_bytes<float>(nf) : sweep_smem_bytes<double>(nf);
  return smem <= 227 * 1024;
}

cudaError_t sweep_prepare(SweepPlan& plan, void* const f[2][4], void* const w[2][4], int64_t N, int nf,
                          int prec, int device) {
  const bool f32 = prec == CE_F32;
  const size_t es = f32 ? 4 : 8;
  plan.tx = f32 ? 128 : 64;
  plan.ty = kTY;
  plan.threads = 32 * kTY;
  plan.stages = kStages;
  plan.smem = f32 ? sweep_smem_bytes<float>(nf) : sweep_smem_bytes<double>(nf);
  const void* kern = f32 ? sweep_kernel_ptr<float>(nf) : sweep_kernel_ptr<double>(nf);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, plan.threads, plan.smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  plan.blocks_per_sm = per_sm;
  plan.gx = (int)(N / plan.tx);
  plan.gy = (int)(N / plan.ty);
  // z chunks: balance whole waves of resident CTAs against the 2 extra planes
  // each chunk loads.
  const double wave = (double)per_sm * sms;
  double best = 1e30;
  int best_gz = 1;
  for (int gz = 1; gz <= N / 4 && gz <= 256; ++gz) {
    const double nblk = (double)plan.gx * plan.gy * gz;
    const double waves = std::ceil(nblk / wave);
    const double eff = nblk / (waves * wave);
    const double tz = (double)N / gz;
    const double cost = (1.0 / eff) * (tz + 2.0) / tz;
    if (cost < best - 1e-9) {
      best = cost;
      best_gz = gz;
    }
  }
  plan.gz = best_gz;

  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t gdim[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)N};
  const cuuint64_t gstride[2] = {(cuuint64_t)(N * es), (cuuint64_t)(N * N * es)};
  const cuuint32_t estride[3] = {1, 1, 1};
  const cuuint32_t rows[3] = {(cuuint32_t)kTY + 2, (cuuint32_t)kTY + 1, 1};
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < nf; ++i)
      for (int a = 0; a < 2; ++a) {
        void* base = a == 0 ? f[b][i] : w[b][i];
        for (int k = 0; k < 3; ++k) {
          const cuuint32_t box[3] = {(cuuint32_t)plan.tx, rows[k], 1};
          CUresult r = enc(&plan.maps[b].m[i][a][k],
                           f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, base,
                           gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
          if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        }
      }
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_step_sweep(const StepArgs<T>& a, const SweepPlan& plan, cudaStream_t st) {
  const dim3 grid(plan.gx, plan.gy, plan.gz);
  const SweepMaps& m = plan.maps[a.in_slot];
  switch (a.nf) {
    case 1: k_step_sweep<T, 1, kTY, kStages><<<grid, plan.threads, plan.smem, st>>>(a, m); break;
    case 2: k_step_sweep<T, 2, kTY, kStages><<<grid, plan.threads, plan.smem, st>>>(a, m); break;
    case 3: k_step_sweep<T, 3, kTY, kStages><<<grid, plan.threads, plan.smem, st>>>(a, m); break;
    default: k_step_sweep<T, 4, kTY, kStages><<<grid, plan.threads, plan.smem, st>>>(a, m); break;
  }
  return cudaGetLastError();
}
template cudaError_t launch_step_sweep<float>(const StepArgs<float>&, const SweepPlan&, cudaStream_t);
template cudaError_t launch_step_sweep<double>(const StepArgs<double>&, const SweepPlan&, cudaStream_t);

}  // namespace ce
