// ce_sweep3d_f32.cu -- instantiations of the 3D z-sweep step kernel for float
// storage (every compiled (rows, stages) variant and field count); kept apart
// from the double instantiations so the two compile in parallel.
#include "ce_sweep3d.cuh"

namespace ce {
namespace sweep {
namespace {

static_assert(kNumVariants == 6, "the switches below cover every compiled variant");

template <int NF, int V>
cudaError_t launch_v(const StepArgs<float>& a, const SweepMaps& m, dim3 grid, size_t smem, cudaStream_t st) {
  constexpr int TY = kVariants[V].ty, NST = kVariants[V].stages;
  k_step_sweep<float, NF, TY, NST><<<grid, 32 * (TY + 1), smem, st>>>(a, m);
  return cudaGetLastError();
}

template <int NF, int V>
const void* kptr_v() {
  constexpr int TY = kVariants[V].ty, NST = kVariants[V].stages;
  return reinterpret_cast<const void*>(&k_step_sweep<float, NF, TY, NST>);
}

template <int NF>
cudaError_t launch_nf(int v, const StepArgs<float>& a, const SweepMaps& m, dim3 g, size_t smem, cudaStream_t st) {
  switch (v) {
    case 0: return launch_v<NF, 0>(a, m, g, smem, st);
    case 1: return launch_v<NF, 1>(a, m, g, smem, st);
    case 2: return launch_v<NF, 2>(a, m, g, smem, st);
    case 3: return launch_v<NF, 3>(a, m, g, smem, st);
    case 4: return launch_v<NF, 4>(a, m, g, smem, st);
    default: return launch_v<NF, 5>(a, m, g, smem, st);
  }
}

template <int NF>
const void* kptr_nf(int v) {
  switch (v) {
    case 0: return kptr_v<NF, 0>();
    case 1: return kptr_v<NF, 1>();
    case 2: return kptr_v<NF, 2>();
    case 3: return kptr_v<NF, 3>();
    case 4: return kptr_v<NF, 4>();
    default: return kptr_v<NF, 5>();
  }
}

}  // namespace

cudaError_t launch_f32(int variant, const StepArgs<float>& a, const SweepMaps& m, dim3 grid, size_t smem,
                       cudaStream_t st) {
  switch (a.nf) {
    case 1: return launch_nf<1>(variant, a, m, grid, smem, st);
    case 2: return launch_nf<2>(variant, a, m, grid, smem, st);
    case 3: return launch_nf<3>(variant, a, m, grid, smem, st);
    default: return launch_nf<4>(variant, a, m, grid, smem, st);
  }
}

const void* kernel_f32(int variant, int nf) {
  switch (nf) {
    case 1: return kptr_nf<1>(variant);
    case 2: return kptr_nf<2>(variant);
    case 3: return kptr_nf<3>(variant);
    default: return kptr_nf<4>(variant);
  }
}

}  // namespace sweep
}  // namespace ce
