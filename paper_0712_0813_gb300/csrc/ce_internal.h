// ce_internal.h -- structures shared by the host side of the C ABI and the
// kernels of libclusterlat.  Not part of the public interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>
#include <cuda.h>
#include <cuda_runtime.h>

#include "clusterlat.h"

namespace ce {

// Scale-factor state belonging to one integer time t_n.  Two slots alternate
// between step launches (launch k reads slot k%2 and writes slot (k+1)%2), so a
// launch never overwrites what its own blocks are still reading.
//
// The velocity state kept in HBM is w with  f'(t_n + dt/2) = w + c f(t_n).  The
// fused step kernel cannot add the expansion term (a''/a) f of its own kick,
// because a'' needs the global sums of the f it is writing; that term is folded
// in by the next launch through c = dt a''/a (and c = 0 after a restore).
struct DevScalars {
  double a;    // a(t_n)
  double ap;   // a'(t_n + dt/2)
  double app;  // a''(t_n)
  double s;    // a''(t_n) / a(t_n)
  double c;    // coefficient of f in the velocity reconstruction above
  double G;    // mean gradient energy of f(t_n) (when computed by a step)
  double V;    // mean potential energy of f(t_n)
  double pad;
};

constexpr int kResultLen = 64;

// Result layout of the diagnostics pass (doubles).
enum ResultIndex : int {
  R_K = 0,       // 4: <1/2 u_i^2>
  R_G = 4,       // 4: gradient energy per field
  R_V = 8,
  R_E = 9,
  R_A = 10,
  R_AP = 11,     // a'(t) at integer time
  R_RESID = 12,
  R_MEAN = 13,   // 4
  R_VAR = 17,    // 4
  R_KTOT = 21,
  R_GTOT = 22,
};

struct DevAux {
  DevScalars slot[2];
  int status;              // CE_OK or the first device-side error code
  unsigned int counter;    // last-block-done counter of the step reduction
  unsigned int counter_diag;
  int pad;
  double result[kResultLen];
};

// Arguments of one step launch.  T is the storage/arithmetic type of fields
// and velocities; the global sums and scalars are always double.
template <typename T>
struct StepArgs {
  const T* f_in[4];
  const T* w_in[4];
  T* f_out[4];
  T* w_out[4];
  int64_t N;
  int64_t S;
  int dims;
  int nf;
  T inv_dx2;
  T dt_drift;      // dt for a step, 0 for the start-up half kick
  T dt_kick;       // dt for a step, dt/2 for the start-up half kick
  T q[3];
  double dt;
  double kappa2;
  double inv_S;
  double half_inv_dx2;
  int update_scalars;   // 1: reduce G, V and advance a, a', a'' in the last block
  int in_slot;          // which ping-pong buffer set is the input (selects TMA maps)
  long long wait_cycles;      // bound of every mbarrier wait (SM clock cycles)
  unsigned int missing_tx;    // test-only: bytes announced per plane that never arrive
  const DevScalars* sc_in;
  DevScalars* sc_out;
  double* partials;     // >= 2 * number of blocks
  unsigned int* counter;
  int* status;
};

// Arguments of the diagnostics pass (energies, moments, synchronised u).
template <typename T>
struct DiagArgs {
  const T* f[4];
  const T* w[4];
  int64_t N;
  int64_t S;
  int dims;
  int nf;
  double inv_dx2;
  double dt;
  double q[3];
  double kappa2;
  int expansion;
  int raw_u;            // 1: w holds u itself (start-up input), no correction
  const DevScalars* sc;
  double* partials;     // nvals * blocks
  DevAux* aux;
  double* u_out;        // sync_u_range only: u of sites [s0, s0 + count)
  int64_t s0;
  int64_t count;
};

// ---- launchers (return cudaError_t of the launch) -------------------------
template <typename T> cudaError_t launch_step_generic(const StepArgs<T>& a, int blocks, cudaStream_t st);
template <typename T> cudaError_t launch_diag(const DiagArgs<T>& a, int blocks, cudaStream_t st);
template <typename T> cudaError_t launch_sync_u_range(const DiagArgs<T>& a, cudaStream_t st);
cudaError_t launch_init_scalars(DevAux* aux, int cur, int expansion, double dt, double kappa2,
                                cudaStream_t st);
template <typename T> cudaError_t launch_from_f64(const double* src, T* dst, int64_t n, cudaStream_t st);
template <typename T> cudaError_t launch_to_f64(const T* src, double* dst, int64_t n, cudaStream_t st);
template <typename T> cudaError_t launch_vhalf_to_f64(const T* f, const T* w, const DevScalars* sc,
                                                      double* dst, int64_t n, cudaStream_t st);

// 3D z-sweep kernel (sm_103a).  TMA tensor maps of the input arrays, per
// field and array (0 = f, 1 = w), for the four boxes the kernel loads:
// TX x (TY+2) rows (interior tile), TX x (TY+1) (tile at the y edge), TX x 1
// (the wrapped halo row), 16 bytes x TY (an x-halo column).  One set per
// ping-pong input buffer.
struct SweepMaps {
  CUtensorMap m[4][2][4];
};
struct SweepPlan {
  int variant;            // index into the compiled (rows, stages) variants
  int tx, ty;             // tile extents in x and y (sites)
  int gx, gy, gz;         // grid: x tiles, y tiles, z chunks
  int threads;
  int stages;
  int blocks_per_sm;
  size_t smem;
  SweepMaps maps[2];
};
bool sweep_supported(int dims, int64_t N, int nf, int prec);
// Whether some compiled variant matches the hints (0 = any).
bool sweep_hint_valid(int64_t N, int nf, int prec, int rows, int stages);
// Pick the variant (hints 0 = automatic), the grid and the z-chunks, and
// encode the tensor maps of the state buffers.  Returns a cudaError_t
// (cudaErrorNotSupported if the driver lacks tensor-map encoding).
cudaError_t sweep_prepare(SweepPlan& plan, void* const f[2][4], void* const w[2][4], int64_t N, int nf,
                          int prec, int device, int rows_hint, int stages_hint, int zchunks_hint);
template <typename T> cudaError_t launch_step_sweep(const StepArgs<T>& a, const SweepPlan& plan,
                                                    cudaStream_t st);
// 3D column kernel with plain loads (any N): warps over strips of 30 x-sites
// by a group of ty rows, 4 warps per block, z-chunks of zlen planes.
struct ColsPlan {
  int nstrips, ngroups, gx, gz, zlen, ty;
};
ColsPlan cols_plan(int64_t N, int nf, int prec, int sms);
template <typename T> cudaError_t launch_step_cols(const StepArgs<T>& a, const ColsPlan& plan, cudaStream_t st);
// 2D line-sweep kernel with plain loads (any N): blocks of 8 strips of 30
// sites in x, y-chunks of ylen rows.
struct LinesPlan {
  int nstrips, gx, gy, ylen;
};
LinesPlan lines_plan(int64_t N, int nf, int prec, int sms);
template <typename T> cudaError_t launch_step_lines(const StepArgs<T>& a, const LinesPlan& plan,
                                                    cudaStream_t st);
namespace sweep {
cudaError_t launch_f32(int variant, const StepArgs<float>& a, const SweepMaps& m, dim3 grid, size_t smem,
                       cudaStream_t st);
cudaError_t launch_f64(int variant, const StepArgs<double>& a, const SweepMaps& m, dim3 grid, size_t smem,
                       cudaStream_t st);
const void* kernel_f32(int variant, int nf);
const void* kernel_f64(int variant, int nf);
}  // namespace sweep

}  // namespace ce

struct ce_batch;

// A simulation handle (opaque in the public header).
struct ce_sim {
  ce_config cfg;
  int dims = 0, nf = 0, prec = CE_F64;
  int64_t N = 0, S = 0;
  size_t esize = 8;
  double dx = 0.0, kappa2 = 0.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  void* f[2][4] = {};
  void* w[2][4] = {};
  ce::DevAux* aux = nullptr;
  double* partials = nullptr;
  double* staging = nullptr;    // chunk x nf doubles, used as two halves by the transfers
  int64_t chunk = 0;
  cudaStream_t xfer = nullptr;  // host <-> device copies of the pipelined transfers
  cudaEvent_t xready[2] = {nullptr, nullptr}, xfree[2] = {nullptr, nullptr}, xstart = nullptr;
  int cur = 0;
  bool have_state = false;
  double t = 0.0;
  int64_t step = 0;
  int kernel = CE_KERNEL_GENERIC;
  int sms = 1;                 // streaming multiprocessors of the handle's device
  int generic_blocks = 1;
  int diag_blocks_max = 8;     // grid cap of the diagnostics pass: 8 blocks per SM
  ce::SweepPlan plan{};
  ce::ColsPlan cols{};
  ce::LinesPlan lines{};
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // kGraphSteps steps starting from buffer set 0 / 1
  bool graphs_ok = true;
  int64_t bytes = 0;
  ce_batch* batch = nullptr;   // set while the handle is a member of a batch
  ce_batch* rows = nullptr;    // private one-lattice batch (CE_KERNEL_ROWS)
  struct Alloc {
    void* p;
    size_t n;
  };
  std::vector<Alloc> allocs;
};

namespace ce {

// Set the thread-local message returned by ce_last_error().
void set_last_error(const std::string& msg);

// Wait until the batch a handle belongs to has finished its queued steps.
cudaError_t batch_wait(ce_batch* b);
// A member is being freed: finish the batch's work and mark the batch unusable.
void batch_detach(ce_batch* b, ce_sim* s);
// Release the output work buffers (spectrum plan, arrays) of a handle.
void outputs_release(const ce_sim* s);
// The batched kernel on one handle (CE_KERNEL_ROWS): build, launch one step
// reading buffer set `in`, release.
int rows_create(ce_sim* s, ce_batch** out);
cudaError_t rows_launch(const ce_batch* b, int in, cudaStream_t st);
void rows_free(ce_batch* b);

constexpr int kGenericThreads = 256;
// Grid of the generic kernel: one thread per site, at most 8 blocks per SM.
int generic_blocks(int64_t S, int sms);
// Streaming multiprocessors of a device (device < 0: the current one), read
// once per device from cudaDevAttrMultiProcessorCount; 1 if it cannot be read.
int sm_count(int device);

}  // namespace ce
