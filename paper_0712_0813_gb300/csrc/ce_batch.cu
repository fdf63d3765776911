// ce_batch.cu -- one leapfrog step of many lattices (any mix of 1D/2D/3D and
// sizes) in a single persistent launch, and the ce_batch_* C ABI around it.
//
// Per site the arithmetic is the fused step of the single-lattice kernels
// (arXiv:0712.0813 Sec. III staggered leapfrog): v = w + c f, g = f + dt v,
// w_out = v + dt (lap g - dV/df(g)), f_out = g, plus the sums of
// (g(x+e_d) - g(x))^2 and V(g) that advance each lattice's own scale factor.
//
// Work decomposition.  Every lattice of the batch is cut into work items of
// about the same size: a CTA of 8 warps takes one item; each warp owns one row
// segment of 32 lanes x VX consecutive x-sites (VX = 16 B / sizeof(T)) and
// sweeps it along the slowest axis (z in 3D, y in 2D; 1D items have no sweep).
// Sweep-axis neighbours stay in registers (own rows are prefetched one plane
// ahead), x-neighbours come from the adjacent lane by shuffle and from plain
// loads at the segment ends, the y-neighbour rows of a 3D plane are the
// neighbouring warps' own rows and are served by L1.  Segments may be partial
// (N not a multiple of 32 VX): lanes past the row end idle.
//
// The grid is persistent: a fixed number of resident CTAs pull items from one
// queue (an atomic counter), largest items first.  The CTA that completes the
// last item of a lattice combines that lattice's item partials in item order
// and advances its a, a', a'' -- nobody waits for anybody.  The last CTA to
// leave resets the queue for the next launch.  One launch advances every
// lattice by one step; step loops are CUDA graphs of 32 launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "ce_device.cuh"
#include "ce_internal.h"

namespace ce {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kBatchGraphSteps = 32;

template <typename T>
struct BMember {
  T* f[2][4];
  T* w[2][4];
  DevScalars* slot;        // the lattice's two scalar slots
  int* status;
  unsigned int* done;      // items of this lattice completed in the running launch
  double* partials;        // 2 doubles per item of this lattice
  int dims, N, p0, first_item, n_items, update_scalars;
  T inv_dx2, dt, q[3];
  double ddt, kappa2, inv_S, half_inv_dx2;
};

struct BItem {
  int member;
  int x0;      // first x site of the (first) segment
  int y0;      // first row (3D items)
  int s0, s1;  // sweep range: z (3D), y (2D); [0, 1) for 1D
};

template <typename T, int VX>
__device__ __forceinline__ void ld16(const T* p, T (&o)[VX]) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = v.x; o[1] = v.y;
  }
}

template <typename T, int VX>
__device__ __forceinline__ void st16(T* p, const T (&o)[VX]) {
  if constexpr (sizeof(T) == 4) {
    __stcs(reinterpret_cast<float4*>(p), make_float4(o[0], o[1], o[2], o[3]));
  } else {
    __stcs(reinterpret_cast<double2*>(p), make_double2(o[0], o[1]));
  }
}

// One warp's row segment of an item.  DIMS 3: row y, sweep z.  DIMS 2: sweep
// y.  DIMS 1: a single "plane".
template <typename T, int NF, int DIMS>
__device__ __forceinline__ void warp_segment(const BMember<T>* __restrict__ m, int in, int x0, int y, int s0,
                                             int s1, int lane, T& g2loc, T& vloc) {
  constexpr int VX = 16 / sizeof(T);
  const int N = m->N;
  const int64_t NN = (int64_t)N * N;
  const int nvl = min(32, (N - x0) / VX);  // valid lanes of this segment
  const bool valid = lane < nvl;
  const int col = x0 + lane * VX;
  const int xl = (x0 == 0) ? N - 1 : x0 - 1;
  const int xr = (x0 + nvl * VX == N) ? 0 : x0 + nvl * VX;
  const bool need_l = (lane == 0), need_r = (lane == nvl - 1);
  const int64_t sweep_stride = DIMS == 3 ? NN : (DIMS == 2 ? (int64_t)N : 0);
  const int64_t row_base = DIMS == 3 ? (int64_t)y * N : 0;
  const int64_t ym_base = DIMS == 3 ? (int64_t)(y == 0 ? N - 1 : y - 1) * N : 0;
  const int64_t yp_base = DIMS == 3 ? (int64_t)(y == N - 1 ? 0 : y + 1) * N : 0;
  const T c = (T)m->slot[in].c;
  const T dd = m->dt, kk = m->dt, idx2 = m->inv_dx2;
  T q[3] = {m->q[0], m->q[1], m->q[2]};
  const T* fi[NF];
  const T* wi[NF];
  T* fo[NF];
  T* wo[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    fi[i] = m->f[in][i];
    wi[i] = m->w[in][i];
    fo[i] = m->f[in ^ 1][i];
    wo[i] = m->w[in ^ 1][i];
  }
  auto wrap = [&](int s) { return s < 0 ? s + N : (s >= N ? s - N : s); };
  auto own = [&](int s, T (&f)[NF][VX], T (&w)[NF][VX]) {
    const int64_t o = row_base + (int64_t)wrap(s) * sweep_stride + col;
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      if (valid) {
        ld16<T, VX>(fi[i] + o, f[i]);
        ld16<T, VX>(wi[i] + o, w[i]);
      } else {
#pragma unroll
        for (int j = 0; j < VX; ++j) f[i][j] = w[i][j] = T(0);
      }
    }
  };
  auto gval = [&](T f, T w) { return fmaT(dd, fmaT(c, f, w), f); };

  T gp[NF][VX], gc[NF][VX], vc[NF][VX], pf[NF][VX], pw[NF][VX];
  if constexpr (DIMS >= 2) {
    own(s0 - 1, pf, pw);
#pragma unroll
    for (int i = 0; i < NF; ++i)
#pragma unroll
      for (int j = 0; j < VX; ++j) gp[i][j] = gval(pf[i][j], pw[i][j]);
  }
  own(s0, pf, pw);
#pragma unroll
  for (int i = 0; i < NF; ++i)
#pragma unroll
    for (int j = 0; j < VX; ++j) {
      vc[i][j] = fmaT(c, pf[i][j], pw[i][j]);
      gc[i][j] = fmaT(dd, vc[i][j], pf[i][j]);
    }
  if constexpr (DIMS >= 2) own(s0 + 1, pf, pw);

  for (int s = s0; s < s1; ++s) {
    T gn[NF][VX], vn[NF][VX];
    if constexpr (DIMS >= 2) {
#pragma unroll
      for (int i = 0; i < NF; ++i)
#pragma unroll
        for (int j = 0; j < VX; ++j) {
          vn[i][j] = fmaT(c, pf[i][j], pw[i][j]);
          gn[i][j] = fmaT(dd, vn[i][j], pf[i][j]);
        }
      if (s + 2 <= s1) own(s + 2, pf, pw);  // prefetch two planes ahead of s
    }
    const int64_t here = row_base + (int64_t)s * sweep_stride;
    T lap[NF][VX];
#pragma unroll
    for (int i = 0; i < NF; ++i) {
      T ym[VX], yp[VX];
      if constexpr (DIMS == 3) {
        T f[VX], w[VX];
        if (valid) {
          ld16<T, VX>(fi[i] + ym_base + (int64_t)s * NN + col, f);
          ld16<T, VX>(wi[i] + ym_base + (int64_t)s * NN + col, w);
#pragma unroll
          for (int j = 0; j < VX; ++j) ym[j] = gval(f[j], w[j]);
          ld16<T, VX>(fi[i] + yp_base + (int64_t)s * NN + col, f);
          ld16<T, VX>(wi[i] + yp_base + (int64_t)s * NN + col, w);
#pragma unroll
          for (int j = 0; j < VX; ++j) yp[j] = gval(f[j], w[j]);
        } else {
#pragma unroll
          for (int j = 0; j < VX; ++j) ym[j] = yp[j] = T(0);
        }
      }
      const int64_t hrow = row_base + (int64_t)s * sweep_stride;
      T hlv = T(0), hrv = T(0);
      if (need_l) hlv = gval(__ldg(fi[i] + hrow + xl), __ldg(wi[i] + hrow + xl));
      if (need_r) hrv = gval(__ldg(fi[i] + hrow + xr), __ldg(wi[i] + hrow + xr));
      T gl = __shfl_up_sync(0xffffffffu, gc[i][VX - 1], 1);
      T gr = __shfl_down_sync(0xffffffffu, gc[i][0], 1);
      if (need_l) gl = hlv;
      if (need_r) gr = hrv;
#pragma unroll
      for (int j = 0; j < VX; ++j) {
        const T g = gc[i][j];
        const T xm = (j == 0) ? gl : gc[i][j - 1];
        const T xp = (j == VX - 1) ? gr : gc[i][j + 1];
        T acc = T(0);
        acc += (xp + xm) - T(2) * g;
        T d2 = (xp - g) * (xp - g);
        if constexpr (DIMS == 3) {
          acc += (yp[j] + ym[j]) - T(2) * g;
          acc += (gn[i][j] + gp[i][j]) - T(2) * g;
          d2 = fmaT(yp[j] - g, yp[j] - g, d2);
          d2 = fmaT(gn[i][j] - g, gn[i][j] - g, d2);
        } else if constexpr (DIMS == 2) {
          acc += (gn[i][j] + gp[i][j]) - T(2) * g;
          d2 = fmaT(gn[i][j] - g, gn[i][j] - g, d2);
        }
        lap[i][j] = acc * idx2;
        if (valid) g2loc += d2;
      }
    }
#pragma unroll
    for (int j = 0; j < VX; ++j) {
      T gs[NF], dv[NF], vs;
#pragma unroll
      for (int i = 0; i < NF; ++i) gs[i] = gc[i][j];
      model_dv<T, NF>(gs, q, dv, vs);
      if (valid) vloc += vs;
#pragma unroll
      for (int i = 0; i < NF; ++i) lap[i][j] = fmaT(kk, lap[i][j] - dv[i], vc[i][j]);
    }
    if (valid) {
#pragma unroll
      for (int i = 0; i < NF; ++i) {
        st16<T, VX>(fo[i] + here + col, gc[i]);
        st16<T, VX>(wo[i] + here + col, lap[i]);
      }
    }
    if constexpr (DIMS >= 2) {
#pragma unroll
      for (int i = 0; i < NF; ++i)
#pragma unroll
        for (int j = 0; j < VX; ++j) {
          gp[i][j] = gc[i][j];
          gc[i][j] = gn[i][j];
          vc[i][j] = vn[i][j];
        }
    }
  }
}

template <typename T, int NF>
__global__ void __launch_bounds__(kThreads) k_step_batched(const BMember<T>* __restrict__ members,
                                                            const BItem* __restrict__ items, int n_items,
                                                            unsigned int* queue, int par) {
  constexpr int VX = 16 / sizeof(T);
  __shared__ int s_item;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(&queue[0], 1u);
    __syncthreads();
    const int itx = s_item;
    if (itx >= n_items) break;
    const BItem it = items[itx];
    const BMember<T>* m = members + it.member;
    const int in = m->p0 ^ par;
    T g2loc = T(0), vloc = T(0);
    if (m->dims == 3) {
      const int y = it.y0 + warp;
      if (y < m->N) warp_segment<T, NF, 3>(m, in, it.x0, y, it.s0, it.s1, lane, g2loc, vloc);
    } else {
      const int x0 = it.x0 + warp * 32 * VX;
      if (x0 < m->N) {
        if (m->dims == 2) warp_segment<T, NF, 2>(m, in, x0, 0, it.s0, it.s1, lane, g2loc, vloc);
        else warp_segment<T, NF, 1>(m, in, x0, 0, 0, 1, lane, g2loc, vloc);
      }
    }
    if (m->update_scalars) {
      double g2 = (double)g2loc, pot = (double)vloc;
      block_sum2(g2, pot);
      if (threadIdx.x == 0) {
        const int k = itx - m->first_item;
        m->partials[2 * k] = g2;
        m->partials[2 * k + 1] = pot;
        __threadfence();
        if (atomicAdd(m->done, 1u) == (unsigned int)(m->n_items - 1)) {
          // last item of this lattice: combine in item order, advance a
          __threadfence();
          double G = 0.0, V = 0.0;
          for (int j = 0; j < m->n_items; ++j) {
            G += __ldcg(m->partials + 2 * j);
            V += __ldcg(m->partials + 2 * j + 1);
          }
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
  double* d_partials = nullptr;      // 2 per item
  int n_items = 0, blocks = 0, par = 0, sweep_len = 32;
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

template <typename T, int NF>
cudaError_t launch_nf(const ce_batch* b, int par) {
  ce::k_step_batched<T, NF><<<b->blocks, ce::kThreads, 0, b->stream>>>(
      static_cast<const ce::BMember<T>*>(b->d_members), static_cast<const ce::BItem*>(b->d_items), b->n_items,
      b->d_queue, par);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_t(const ce_batch* b, int par) {
  switch (b->nf) {
    case 1: return launch_nf<T, 1>(b, par);
    case 2: return launch_nf<T, 2>(b, par);
    case 3: return launch_nf<T, 3>(b, par);
    default: return launch_nf<T, 4>(b, par);
  }
}

cudaError_t launch_batch(const ce_batch* b, int par) {
  return b->prec == CE_F32 ? launch_t<float>(b, par) : launch_t<double>(b, par);
}

const void* batch_kernel(int prec, int nf) {
  if (prec == CE_F32) {
    switch (nf) {
      case 1: return (const void*)&ce::k_step_batched<float, 1>;
      case 2: return (const void*)&ce::k_step_batched<float, 2>;
      case 3: return (const void*)&ce::k_step_batched<float, 3>;
      default: return (const void*)&ce::k_step_batched<float, 4>;
    }
  }
  switch (nf) {
    case 1: return (const void*)&ce::k_step_batched<double, 1>;
    case 2: return (const void*)&ce::k_step_batched<double, 2>;
    case 3: return (const void*)&ce::k_step_batched<double, 3>;
    default: return (const void*)&ce::k_step_batched<double, 4>;
  }
}

// Cut every member into items of about kWarps x 32 x VX x sweep_len sites.
template <typename T>
void build_tables(ce_batch* b, std::vector<ce::BMember<T>>& mem, std::vector<ce::BItem>& items) {
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
      for (int x0 = 0; x0 < N; x0 += SEG)
        for (int y0 = 0; y0 < N; y0 += ce::kWarps)
          for (int z0 = 0; z0 < N; z0 += L)
            add(x0, y0, z0, std::min(N, z0 + L), (int64_t)std::min(SEG, N - x0) * std::min(ce::kWarps, N - y0) * (std::min(N, z0 + L) - z0));
    } else if (s->dims == 2) {
      for (int x0 = 0; x0 < N; x0 += ce::kWarps * SEG)
        for (int y0 = 0; y0 < N; y0 += L)
          add(x0, 0, y0, std::min(N, y0 + L), (int64_t)std::min(ce::kWarps * SEG, N - x0) * (std::min(N, y0 + L) - y0));
    } else {
      for (int x0 = 0; x0 < N; x0 += ce::kWarps * SEG) add(x0, 0, 0, 1, (int64_t)std::min(ce::kWarps * SEG, N - x0));
    }
  }
  // items of a member stay contiguous (their partials are indexed from first_item);
  // members are ordered by their largest item so the queue hands out big work first
  std::vector<size_t> order(b->members.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) {
    return per[a].front().cost * (int64_t)per[a].size() > per[c].front().cost * (int64_t)per[c].size();
  });
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
    m.p0 = s->cur ^ b->par;
    m.first_item = (int)items.size();
    m.n_items = (int)per[k].size();
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

template <typename T>
int upload_tables(ce_batch* b) {
  std::vector<ce::BMember<T>> mem;
  std::vector<ce::BItem> items;
  // partial-sum slots are assigned after the item count is known
  build_tables<T>(b, mem, items);
  b->n_items = (int)items.size();
  cudaError_t e = cudaMalloc(&b->d_partials, sizeof(double) * 2 * std::max(1, b->n_items));
  if (e != cudaSuccess) return bcuda(e, "ce_batch_create: partials");
  for (auto& m : mem) m.partials = b->d_partials + 2 * (int64_t)m.first_item;
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
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

cudaError_t ensure_batch_graph(ce_batch* b, int start) {
  if (b->graph[start]) return cudaSuccess;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  cudaError_t el = cudaSuccess;
  int par = start;
  for (int k = 0; k < ce::kBatchGraphSteps && el == cudaSuccess; ++k) {
    el = launch_batch(b, par);
    par ^= 1;
  }
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

void ce::batch_detach(ce_batch* b, ce_sim* s) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& m : b->members)
    if (m == s) m = nullptr;
  b->broken = true;
}

extern "C" {

int ce_batch_create(ce_sim* const* sims, int n, int sweep_len, void* stream, ce_batch** out) {
  ce::set_last_error("");
  if (!out) return bfail(CE_EINVAL, "ce_batch_create: out is NULL");
  *out = nullptr;
  if (!sims || n < 1) return bfail(CE_EINVAL, "ce_batch_create: need at least one simulation");
  if (sweep_len < 0 || sweep_len > 4096) return bfail(CE_EINVAL, "ce_batch_create: sweep_len must be 0..4096");
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
  b->sweep_len = sweep_len > 0 ? sweep_len : 32;
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
  const void* kern = batch_kernel(b->prec, b->nf);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, ce::kThreads, 0);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e != cudaSuccess || per_sm < 1) {
    release(b);
    delete b;
    return bcuda(e != cudaSuccess ? e : cudaErrorInvalidConfiguration, "ce_batch_create: occupancy");
  }
  b->blocks = std::max(1, std::min(per_sm * sms, b->n_items));
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
  for (int64_t k = 0; k < n; ++k) {
    e = launch_batch(b, b->par);
    if (e != cudaSuccess) return bcuda(e, "ce_batch_step: launch");
    b->par ^= 1;
    advance_members(b, 1);
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

int ce_batch_info(const ce_batch* b, int* members, int* items, int* blocks, int64_t* sites) {
  if (!b || !members || !items || !blocks || !sites) return bfail(CE_EINVAL, "ce_batch_info: NULL argument");
  *members = (int)b->members.size();
  *items = b->n_items;
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
