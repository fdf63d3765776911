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
#include "ce_plan.h"
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
    plan.gz = plan::auto_zchunks(N, (int64_t)plan.gx * plan.gy, per_sm, sms);   // ce_plan.h
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
