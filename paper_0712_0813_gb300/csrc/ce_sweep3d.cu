// ce_sweep3d.cu -- host side of the 3D z-sweep step kernel: which variants
// apply to a lattice, the launch plan (variant, grid, z-chunks), the TMA tensor
// maps of the state buffers, and the launch.  The kernel itself is in
// ce_sweep3d.cuh; its instantiations in ce_sweep3d_f32.cu / ce_sweep3d_f64.cu.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <queue>
#include <vector>

#include "ce_internal.h"
#include "ce_sweep3d.cuh"

namespace ce {
namespace {

int tile_x(int prec) { return prec == CE_F32 ? 128 : 64; }

size_t variant_smem(int v, int nf, int prec) {
  const sweep::Variant var = sweep::kVariants[v];
  return prec == CE_F32 ? sweep::smem_bytes<float>(nf, var.ty, var.stages)
                        : sweep::smem_bytes<double>(nf, var.ty, var.stages);
}

bool variant_applies(int v, int64_t N, int nf, int prec) {
  const sweep::Variant var = sweep::kVariants[v];
  const int tx = tile_x(prec);
  if (N % tx != 0 || N % var.ty != 0 || N < 2 * var.ty || N > (1 << 20)) return false;
  return variant_smem(v, nf, prec) <= 227 * 1024;
}

const void* variant_kernel(int v, int nf, int prec) {
  return prec == CE_F32 ? sweep::kernel_f32(v, nf) : sweep::kernel_f64(v, nf);
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

// Predicted duration (in plane-times of a CTA sharing its SM) of a launch of
// cols x gz CTAs, each sweeping its chunk of N / gz planes plus 2 halo planes
// and a start-up of about 4 planes.  Blocks are handed out in grid order to the
// SM slots that free up; a CTA runs 1.32x faster while it is alone on its SM
// (ncu: 2.2k against 2.9k cycles per plane at 256^3), and an SM never streams
// faster than per_sm CTAs sharing it.  The lone-CTA speed-up is what makes a
// partial wave cheaper than a whole one: at 256^3 the model prefers 4 chunks
// (0.84 of a wave; measured 93.3 us) to 14 (101.6 us), which a count of whole
// waves would pick.  Event-driven: one heap entry per SM.
double grid_time(int64_t N, int64_t cols, int gz, int per_sm, int sms) {
  constexpr double kStart = 4.0, kSolo = 1.32;
  const double cap = (double)per_sm;
  auto rate = [&](size_t n) { return std::min(kSolo, cap / (double)n); };
  const int64_t nblk = cols * gz;
  auto work = [&](int64_t b) {
    const int64_t zc = b / cols;
    return (double)((zc + 1) * N / gz - zc * N / gz + 2) + kStart;
  };
  std::vector<std::vector<double>> rem(sms);
  std::vector<double> last(sms, 0.0);
  int64_t next = 0;
  for (int r = 0; r < per_sm; ++r)
    for (int s = 0; s < sms && next < nblk; ++s) rem[s].push_back(work(next++));
  using Ev = std::pair<double, int>;
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> heap;
  for (int s = 0; s < sms; ++s)
    if (!rem[s].empty()) heap.push({*std::min_element(rem[s].begin(), rem[s].end()) / rate(rem[s].size()), s});
  double end = 0.0;
  while (!heap.empty()) {
    const auto [t, s] = heap.top();
    heap.pop();
    const double done = (t - last[s]) * rate(rem[s].size());
    size_t keep = 0, freed = 0;
    for (double w : rem[s]) {
      if (w - done > 1e-9) rem[s][keep++] = w - done;
      else ++freed;
    }
    rem[s].resize(keep);
    for (; freed > 0 && next < nblk; --freed) rem[s].push_back(work(next++));
    last[s] = t;
    end = std::max(end, t);
    if (!rem[s].empty()) heap.push({t + *std::min_element(rem[s].begin(), rem[s].end()) / rate(rem[s].size()), s});
  }
  return end;
}

// Default variant when the caller gives no hint: the first that applies in
// this order of preference.
constexpr int kPreference[] = {0, 1, 3, 2, 4, 5};

}  // namespace

bool sweep_supported(int dims, int64_t N, int nf, int prec) {
  if (dims != 3 || nf < 1 || nf > 4) return false;
  for (int v = 0; v < sweep::kNumVariants; ++v)
    if (variant_applies(v, N, nf, prec)) return true;
  return false;
}

bool sweep_hint_valid(int64_t N, int nf, int prec, int rows, int stages) {
  for (int v = 0; v < sweep::kNumVariants; ++v) {
    const sweep::Variant var = sweep::kVariants[v];
    if ((rows == 0 || rows == var.ty) && (stages == 0 || stages == var.stages) && variant_applies(v, N, nf, prec))
      return true;
  }
  return false;
}

cudaError_t sweep_prepare(SweepPlan& plan, void* const f[2][4], void* const w[2][4], int64_t N, int nf,
                          int prec, int device, int rows_hint, int stages_hint, int zchunks_hint) {
  const bool f32 = prec == CE_F32;
  const size_t es = f32 ? 4 : 8;
  int chosen = -1;
  for (int k = 0; k < sweep::kNumVariants && chosen < 0; ++k) {
    const int v = kPreference[k];
    const sweep::Variant var = sweep::kVariants[v];
    if ((rows_hint == 0 || rows_hint == var.ty) && (stages_hint == 0 || stages_hint == var.stages) &&
        variant_applies(v, N, nf, prec))
      chosen = v;
  }
  if (chosen < 0) return cudaErrorInvalidConfiguration;
  const sweep::Variant var = sweep::kVariants[chosen];
  plan.variant = chosen;
  plan.tx = tile_x(prec);
  plan.ty = var.ty;
  plan.stages = var.stages;
  plan.threads = 32 * (var.ty + 1);
  plan.smem = variant_smem(chosen, nf, prec);
  const void* kern = variant_kernel(chosen, nf, prec);
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
  if (zchunks_hint > 0) {
    if (zchunks_hint > N / 2) return cudaErrorInvalidConfiguration;
    plan.gz = zchunks_hint;
  } else {
    // z-chunks: among chunks of at most 64 planes, the count with the least
    // predicted launch time (grid_time).  Longer chunks measured slower on
    // large lattices than the model says (640^3: 3 chunks 1363 us, 12 chunks
    // 1279 us); with the cap the pick was the measured best, or within 1-5% of
    // it, on every FP32 lattice timed (128^3 to 768^3, 8- and 16-row tiles).
    constexpr int kMaxChunk = 64;
    const int gz_min = (int)std::max<int64_t>(1, (N + kMaxChunk - 1) / kMaxChunk);
    double best = 1e300;
    int best_gz = (int)std::min<int64_t>(gz_min, N / 2);
    for (int gz = gz_min; gz <= N / 4 && gz <= 128; ++gz) {
      if (gz > gz_min && (int64_t)plan.gx * plan.gy * gz > 32LL * per_sm * sms) break;   // 32 waves: no tail left to win
      const double t = grid_time(N, (int64_t)plan.gx * plan.gy, gz, per_sm, sms);
      if (t < best * (1.0 - 1e-6)) {
        best = t;
        best_gz = gz;
      }
    }
    plan.gz = best_gz;
  }

  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encoder();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t gdim[3] = {(cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)N};
  const cuuint64_t gstride[2] = {(cuuint64_t)(N * es), (cuuint64_t)(N * N * es)};
  const cuuint32_t estride[3] = {1, 1, 1};
  // boxes: tile + y halo, tile + one y-halo row (lattice y edge), one row, x-halo column
  const cuuint32_t box_w[4] = {(cuuint32_t)plan.tx, (cuuint32_t)plan.tx, (cuuint32_t)plan.tx, (cuuint32_t)(16 / es)};
  const cuuint32_t box_h[4] = {(cuuint32_t)plan.ty + 2, (cuuint32_t)plan.ty + 1, 1, (cuuint32_t)plan.ty};
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < nf; ++i)
      for (int a = 0; a < 2; ++a) {
        void* base = a == 0 ? f[b][i] : w[b][i];
        for (int k = 0; k < 4; ++k) {
          const cuuint32_t box[3] = {box_w[k], box_h[k], 1};
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

template <>
cudaError_t launch_step_sweep<float>(const StepArgs<float>& a, const SweepPlan& plan, cudaStream_t st) {
  return sweep::launch_f32(plan.variant, a, plan.maps[a.in_slot], dim3(plan.gx, plan.gy, plan.gz), plan.smem, st);
}

template <>
cudaError_t launch_step_sweep<double>(const StepArgs<double>& a, const SweepPlan& plan, cudaStream_t st) {
  return sweep::launch_f64(plan.variant, a, plan.maps[a.in_slot], dim3(plan.gx, plan.gy, plan.gz), plan.smem, st);
}

}  // namespace ce
