// ce_capi.cu -- the extern "C" boundary of libclusterlat (declared in
// include/clusterlat.h): handle lifetime, argument validation, host<->device
// copies, the start-up sequence and the step loop.  All method arithmetic runs
// in the kernels; this file only moves data and sequences launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ce_internal.h"
#include "clusterlat.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return CE_ECUDA;
}

constexpr double kDefaultPhi0OverMpl = 0.342;
constexpr int64_t kMaxSites = int64_t(1) << 34;
constexpr int64_t kStagingChunk = int64_t(1) << 22;   // sites per staging chunk
// Smallest sides for which the automatic FP32 choice takes the row kernel
// (sides that are multiples of 4) and, in 2D, the line-sweep kernel, from
// timings of single lattices (us per step).  3D below side 256 the column
// kernel is as fast or faster than the row kernel (96^3: 16.4 against 19.8,
// 224^3: 77.0 against 81.8, 192^3: 52.7 against 51.5; 288^3: 158.9 against
// 148.9).  2D below side 512 the row kernel and the line-sweep kernel tie
// (512^2: 14.6 both), and below 320 the generic kernel starts faster than the
// line-sweep kernel (257^2: 12.7 against 13.2; 385^2: 15.5 against 12.9).
constexpr int kRowsMinN3 = 256;
constexpr int kRowsMinN2 = 512;
constexpr int kLinesMinN2 = 320;
constexpr int kGraphSteps = 32;   // steps per captured CUDA graph (even: keeps the ping-pong parity)
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: bound of every device-side wait

}  // namespace

void ce::set_last_error(const std::string& msg) { g_err = msg; }


namespace {

void* dalloc(ce_sim* s, size_t n) {
  n = (n + 255) & ~size_t(255);
  void* p = nullptr;
  if (s->cfg.alloc) {
    p = s->cfg.alloc(n, s->stream, s->cfg.alloc_ctx);
  } else if (cudaMalloc(&p, n) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    s->allocs.push_back({p, n});
    s->bytes += (int64_t)n;
  }
  return p;
}

void release_all(ce_sim* s) {
  for (auto& a : s->allocs) {
    if (s->cfg.release) s->cfg.release(a.p, a.n, s->stream, s->cfg.alloc_ctx);
    else if (!s->cfg.alloc) cudaFree(a.p);
  }
  s->allocs.clear();
}

int validate(const ce_config* c, int64_t* S_out) {
  if (!c) return fail(CE_EINVAL, "ce_create: cfg is NULL");
  if (c->dims < 1 || c->dims > 3) return fail(CE_EINVAL, "ce_create: dims must be 1, 2 or 3");
  if (c->N < 3) return fail(CE_EINVAL, "ce_create: N must be >= 3");
  int64_t S = 1;
  for (int d = 0; d < c->dims; ++d) {
    if (S > kMaxSites / c->N) return fail(CE_EINVAL, "ce_create: N^dims exceeds 2^34 sites");
    S *= c->N;
  }
  if (!(c->L > 0.0) || !std::isfinite(c->L)) return fail(CE_EINVAL, "ce_create: L must be finite and > 0");
  if (!(c->dt > 0.0) || !std::isfinite(c->dt)) return fail(CE_EINVAL, "ce_create: dt must be finite and > 0");
  if (c->nfields < 1 || c->nfields > 4) return fail(CE_EINVAL, "ce_create: nfields must be 1..4");
  for (int i = 0; i + 1 < c->nfields; ++i)
    if (!(c->q[i] >= 0.0) || !std::isfinite(c->q[i])) return fail(CE_EINVAL, "ce_create: q_i must be finite and >= 0");
  if (c->precision != CE_F64 && c->precision != CE_F32) return fail(CE_EINVAL, "ce_create: precision must be CE_F64 or CE_F32");
  if (c->kernel < CE_KERNEL_AUTO || c->kernel > CE_KERNEL_PLANES) return fail(CE_EINVAL, "ce_create: unknown kernel");
  if (c->expansion != 0 && c->expansion != 1) return fail(CE_EINVAL, "ce_create: expansion must be 0 or 1");
  if (!!c->alloc != !!c->release) return fail(CE_EINVAL, "ce_create: alloc and release hooks go together");
  if (!std::isfinite(c->phi0_over_mpl) || !std::isfinite(c->phi0)) return fail(CE_EINVAL, "ce_create: non-finite phi0");
  if (c->tile_rows != 0 && c->tile_rows != 4 && c->tile_rows != 8 && c->tile_rows != 16)
    return fail(CE_EINVAL, "ce_create: tile_rows must be 0, 4, 8 or 16");
  if (c->stages != 0 && (c->stages < 3 || c->stages > 5)) return fail(CE_EINVAL, "ce_create: stages must be 0 or 3..5");
  if (c->zchunks < 0 || (c->zchunks > 0 && c->zchunks > c->N / 2))
    return fail(CE_EINVAL, "ce_create: zchunks must be 0 or 1..N/2");
  // Leapfrog stability: dt < 2 / omega_max, omega_max^2 = 4 d / dx^2 + largest mass^2
  // (masses 3 phi0^2 and q_i phi0^2 around the homogeneous phi0).
  if (!(c->flags & CE_FLAG_ALLOW_UNSTABLE_DT)) {
    const double dx = c->L / (double)c->N;
    const double phi0 = c->phi0 > 0.0 ? c->phi0 : 1.0;
    double m2 = 3.0 * phi0 * phi0;
    for (int i = 0; i + 1 < c->nfields; ++i) m2 = std::fmax(m2, c->q[i] * phi0 * phi0);
    const double wmax = std::sqrt(4.0 * c->dims / (dx * dx) + m2);
    if (c->dt >= 2.0 / wmax)
      return fail(CE_EINVAL, "ce_create: dt at or above the leapfrog stability bound 2/omega_max");
  }
  *S_out = S;
  return CE_OK;
}

template <typename T>
ce::StepArgs<T> make_step_args(const ce_sim* s, int in, bool half_kick) {
  ce::StepArgs<T> a{};
  for (int i = 0; i < 4; ++i) {
    const int k = i < s->nf ? i : 0;
    a.f_in[i] = static_cast<const T*>(s->f[in][k]);
    a.w_in[i] = static_cast<const T*>(s->w[in][k]);
    a.f_out[i] = static_cast<T*>(s->f[in ^ 1][k]);
    a.w_out[i] = static_cast<T*>(s->w[in ^ 1][k]);
  }
  a.N = s->N;
  a.S = s->S;
  a.dims = s->dims;
  a.nf = s->nf;
  a.inv_dx2 = (T)(1.0 / (s->dx * s->dx));
  a.dt_drift = half_kick ? T(0) : (T)s->cfg.dt;
  a.dt_kick = half_kick ? (T)(0.5 * s->cfg.dt) : (T)s->cfg.dt;
  for (int i = 0; i < 3; ++i) a.q[i] = (T)s->cfg.q[i];
  a.dt = s->cfg.dt;
  a.kappa2 = s->kappa2;
  a.inv_S = 1.0 / (double)s->S;
  a.half_inv_dx2 = 0.5 / (s->dx * s->dx);
  a.update_scalars = (s->cfg.expansion && !half_kick) ? 1 : 0;
  a.in_slot = in;
  const bool stall = (s->cfg.flags & CE_FLAG_TEST_TMA_STALL) != 0;
  a.wait_cycles = stall ? (1LL << 20) : kWaitCycles;
  a.missing_tx = stall ? 16u : 0u;
  a.sc_in = &s->aux->slot[in];
  a.sc_out = &s->aux->slot[in ^ 1];
  a.partials = s->partials;
  a.counter = &s->aux->counter;
  a.status = &s->aux->status;
  return a;
}

template <typename T>
cudaError_t launch_one_step(const ce_sim* s, int in, bool half_kick) {
  if (s->kernel == CE_KERNEL_ROWS && !half_kick) return ce::rows_launch(s->rows, in, s->stream);
  const ce::StepArgs<T> a = make_step_args<T>(s, in, half_kick);
  if (s->kernel == CE_KERNEL_SWEEP) return ce::launch_step_sweep<T>(a, s->plan, s->stream);
  if (s->kernel == CE_KERNEL_PLANES)
    return s->dims == 3 ? ce::launch_step_cols<T>(a, s->cols, s->stream)
                        : ce::launch_step_lines<T>(a, s->lines, s->stream);
  return ce::launch_step_generic<T>(a, s->generic_blocks, s->stream);
}

cudaError_t step_once(const ce_sim* s, int in, bool half_kick) {
  return s->prec == CE_F32 ? launch_one_step<float>(s, in, half_kick)
                           : launch_one_step<double>(s, in, half_kick);
}

// Capture kGraphSteps consecutive step launches starting from buffer set
// `start` into a CUDA graph (built once per handle and parity, replayed by
// ce_step).  Kernel arguments are fixed per handle, so the graph stays valid
// for the handle's lifetime.
cudaError_t ensure_graph(ce_sim* s, int start) {
  if (s->graph[start]) return cudaSuccess;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  int in = start;
  cudaError_t el = cudaSuccess;
  for (int k = 0; k < kGraphSteps && el == cudaSuccess; ++k) {
    el = step_once(s, in, false);
    in ^= 1;
  }
  e = cudaStreamEndCapture(s->stream, &g);
  if (el != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return el != cudaSuccess ? el : e;
  }
  e = cudaGraphInstantiate(&s->graph[start], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) s->graph[start] = nullptr;
  return e;
}

template <typename T>
ce::DiagArgs<T> make_diag_args(const ce_sim* s, int raw_u) {
  ce::DiagArgs<T> a{};
  for (int i = 0; i < 4; ++i) {
    const int k = i < s->nf ? i : 0;
    a.f[i] = static_cast<const T*>(s->f[s->cur][k]);
    a.w[i] = static_cast<const T*>(s->w[s->cur][k]);
  }
  a.N = s->N;
  a.S = s->S;
  a.dims = s->dims;
  a.nf = s->nf;
  a.inv_dx2 = 1.0 / (s->dx * s->dx);
  a.dt = s->cfg.dt;
  for (int i = 0; i < 3; ++i) a.q[i] = s->cfg.q[i];
  a.kappa2 = s->kappa2;
  a.expansion = s->cfg.expansion;
  a.raw_u = raw_u;
  a.sc = &s->aux->slot[s->cur];
  a.partials = s->partials;
  a.aux = s->aux;
  return a;
}

int diag_blocks(const ce_sim* s) {
  int64_t want = (s->S + 255) / 256;
  return (int)(want < s->diag_blocks_max ? want : s->diag_blocks_max);
}

cudaError_t run_diag(const ce_sim* s, int raw_u) {
  if (s->prec == CE_F32) return ce::launch_diag<float>(make_diag_args<float>(s, raw_u), diag_blocks(s), s->stream);
  return ce::launch_diag<double>(make_diag_args<double>(s, raw_u), diag_blocks(s), s->stream);
}

// Copy the aux block back and turn a latched device error into a return code.
int fetch_aux(ce_sim* s, ce::DevAux* host) {
  cudaError_t e = cudaMemcpyAsync(host, s->aux, sizeof(ce::DevAux), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "device sync");
  if (host->status != CE_OK)
    return fail(host->status, "device reported non-finite global sums or no real a' (fields blew up?)");
  return CE_OK;
}

// Host <-> device transfers through the staging buffer, pipelined: the buffer
// is used as two halves; the handle's stream converts (or computes) one half
// while the transfer stream copies the other, ordered by events (xready[b]:
// half b holds data for its consumer; xfree[b]: its consumer is done with it),
// with one host synchronisation per call instead of one per chunk.  Copies then
// run back to back at the link's bandwidth.

// Sites per half for `rows` values per site.
int64_t half_sites(const ce_sim* s, int rows) {
  return std::max<int64_t>(1, s->chunk * s->nf / (2 * rows));
}

// Host float64 -> device state array (one field).
int upload_field(ce_sim* s, const double* src, void* dst) {
  if (s->prec == CE_F64) {
    cudaError_t e = cudaMemcpyAsync(dst, src, (size_t)s->S * 8, cudaMemcpyHostToDevice, s->stream);
    return e == cudaSuccess ? CE_OK : cuda_fail(e, "H2D copy");
  }
  const int64_t half = half_sites(s, 1);
  // the staging buffer may still be read by earlier work on the handle's stream
  cudaError_t e = cudaEventRecord(s->xstart, s->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s->xfer, s->xstart, 0);
  int k = 0;
  for (int64_t s0 = 0; s0 < s->S && e == cudaSuccess; s0 += half, ++k) {
    const int64_t n = std::min<int64_t>(half, s->S - s0);
    const int b = k & 1;
    double* buf = s->staging + (int64_t)b * half;
    if (k >= 2) e = cudaStreamWaitEvent(s->xfer, s->xfree[b], 0);   // chunk k - 2 converted
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf, src + s0, (size_t)n * 8, cudaMemcpyHostToDevice, s->xfer);
    if (e == cudaSuccess) e = cudaEventRecord(s->xready[b], s->xfer);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->xready[b], 0);
    if (e == cudaSuccess) e = ce::launch_from_f64<float>(buf, static_cast<float*>(dst) + s0, n, s->stream);
    if (e == cudaSuccess) e = cudaEventRecord(s->xfree[b], s->stream);
  }
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s->xfer);   // no copy may still read the caller's buffer after the return
    return cuda_fail(e, "H2D conversion");
  }
  return CE_OK;
}

// Pipelined download of the handle's S sites, `rows` values per site:
// produce(s0, n, buf) launches on the handle's stream the kernel that writes
// rows x n doubles (row-major) for sites s0 .. s0 + n - 1 into buf; row r goes
// to dst + r * S + s0.  Returns after every copy has landed in host memory.
template <typename Produce>
int pipelined_download(ce_sim* s, int rows, double* dst, Produce produce, const char* what) {
  const int64_t half = half_sites(s, rows);
  cudaError_t e = cudaSuccess;
  int k = 0;
  for (int64_t s0 = 0; s0 < s->S && e == cudaSuccess; s0 += half, ++k) {
    const int64_t n = std::min<int64_t>(half, s->S - s0);
    const int b = k & 1;
    double* buf = s->staging + (int64_t)b * half * rows;
    if (k >= 2) e = cudaStreamWaitEvent(s->stream, s->xfree[b], 0);   // chunk k - 2 copied out
    if (e == cudaSuccess) e = produce(s0, n, buf);
    if (e == cudaSuccess) e = cudaEventRecord(s->xready[b], s->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s->xfer, s->xready[b], 0);
    for (int r = 0; r < rows && e == cudaSuccess; ++r)
      e = cudaMemcpyAsync(dst + (int64_t)r * s->S + s0, buf + (int64_t)r * n, (size_t)n * 8, cudaMemcpyDeviceToHost,
                          s->xfer);
    if (e == cudaSuccess) e = cudaEventRecord(s->xfree[b], s->xfer);
  }
  const cudaError_t ex = cudaStreamSynchronize(s->xfer);   // every copy has landed (or failed)
  if (e == cudaSuccess) e = ex;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? CE_OK : cuda_fail(e, what);
}

// Device state array (one field) -> host float64.  With w given, exports
// f'(t+dt/2) = w + c f instead of f.
int download_field(ce_sim* s, const void* f, const void* w, double* dst) {
  if (s->prec == CE_F64 && !w) {
    cudaError_t e = cudaMemcpyAsync(dst, f, (size_t)s->S * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    return e == cudaSuccess ? CE_OK : cuda_fail(e, "D2H copy");
  }
  return pipelined_download(s, 1, dst, [&](int64_t s0, int64_t n, double* buf) -> cudaError_t {
    if (s->prec == CE_F32) {
      const float* fp = static_cast<const float*>(f) + s0;
      return w ? ce::launch_vhalf_to_f64<float>(fp, static_cast<const float*>(w) + s0, &s->aux->slot[s->cur], buf,
                                                n, s->stream)
               : ce::launch_to_f64<float>(fp, buf, n, s->stream);
    }
    const double* fp = static_cast<const double*>(f) + s0;
    return ce::launch_vhalf_to_f64<double>(fp, static_cast<const double*>(w) + s0, &s->aux->slot[s->cur], buf, n,
                                           s->stream);
  }, "D2H conversion");
}

int check_sim(const ce_sim* s, const char* fn) {
  if (!s) return fail(CE_EINVAL, std::string(fn) + ": sim is NULL");
  return CE_OK;
}

// Make the handle's device current and, for a batch member, let the batch's
// queued steps finish first (the member's own stream does not see them).
int select_device(const ce_sim* s) {
  cudaError_t e = cudaSetDevice(s->device);
  if (e == cudaSuccess && s->batch) e = ce::batch_wait(s->batch);
  return e == cudaSuccess ? CE_OK : cuda_fail(e, "cudaSetDevice");
}

}  // namespace

extern "C" {

int ce_version(void) { return 10000; }

const char* ce_last_error(void) { return g_err.c_str(); }

int ce_create(const ce_config* cfg, ce_sim** out) {
  g_err.clear();
  if (!out) return fail(CE_EINVAL, "ce_create: out is NULL");
  *out = nullptr;
  int64_t S = 0;
  int rc = validate(cfg, &S);
  if (rc != CE_OK) return rc;
  const bool sweep_ok = ce::sweep_supported(cfg->dims, cfg->N, cfg->nfields, cfg->precision) &&
                        ce::sweep_hint_valid(cfg->N, cfg->nfields, cfg->precision, cfg->tile_rows, cfg->stages);
  if (cfg->kernel == CE_KERNEL_SWEEP && !sweep_ok)
    return fail(CE_EINVAL, "ce_create: the z-sweep kernel needs dims == 3 and N a multiple of its tile");
  const bool rows_ok = cfg->N % (cfg->precision == CE_F32 ? 4 : 2) == 0;
  if (cfg->kernel == CE_KERNEL_ROWS && !rows_ok)
    return fail(CE_EINVAL, "ce_create: the row kernel needs N a multiple of 4 (FP32) or 2 (FP64)");
  if (cfg->kernel == CE_KERNEL_PLANES && cfg->dims < 2)
    return fail(CE_EINVAL, "ce_create: the plane/line-sweep kernel needs dims 2 or 3");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(CE_ECUDA, std::string("ce_create: no CUDA device (") + cudaGetErrorString(e) + ")");
  }
  ce_sim* s = new (std::nothrow) ce_sim();
  if (!s) return fail(CE_ENOMEM, "ce_create: host allocation failed");
  s->cfg = *cfg;
  s->dims = cfg->dims;
  s->N = cfg->N;
  s->S = S;
  s->nf = cfg->nfields;
  s->prec = cfg->precision;
  s->esize = s->prec == CE_F32 ? 4 : 8;
  s->dx = cfg->L / (double)cfg->N;
  const double p0m = cfg->phi0_over_mpl > 0.0 ? cfg->phi0_over_mpl : kDefaultPhi0OverMpl;
  s->kappa2 = 8.0 * M_PI / 3.0 * p0m * p0m;
  // Automatic choice.  FP32: the z-sweep kernel where it applies, else the row
  // kernel for the 2D and 3D lattices it takes from the sides above, else the
  // column kernel (3D) or the line-sweep kernel (2D) for odd and small sides,
  // else (1D lattices, small 2D sides) the generic kernel.  FP64 is bound by the FP64 rate, and there
  // the generic kernel's two-pass form (each site's g formed once) measured
  // faster than both the z-sweep kernel (256^3: 1090 against 1141 us, tuned
  // plan) and the row kernel (288^3: 1540 against 2967 us): the generic kernel,
  // unless the caller gave z-sweep plan hints.
  const bool sweep_hinted = cfg->tile_rows != 0 || cfg->stages != 0 || cfg->zchunks != 0;
  const bool rows_auto = rows_ok && cfg->precision == CE_F32 && cfg->dims >= 2 &&
                         cfg->N >= (cfg->dims == 3 ? kRowsMinN3 : kRowsMinN2);
  const bool planes_auto = cfg->precision == CE_F32 && (cfg->dims == 3 || (cfg->dims == 2 && cfg->N >= kLinesMinN2));
  if (cfg->kernel == CE_KERNEL_GENERIC) s->kernel = CE_KERNEL_GENERIC;
  else if (cfg->kernel == CE_KERNEL_ROWS) s->kernel = CE_KERNEL_ROWS;
  else if (cfg->kernel == CE_KERNEL_PLANES) s->kernel = CE_KERNEL_PLANES;
  else if (sweep_ok && (cfg->precision == CE_F32 || sweep_hinted || cfg->kernel == CE_KERNEL_SWEEP))
    s->kernel = CE_KERNEL_SWEEP;
  else s->kernel = rows_auto ? CE_KERNEL_ROWS : (planes_auto ? CE_KERNEL_PLANES : CE_KERNEL_GENERIC);
  cudaGetDevice(&s->device);
  s->sms = ce::sm_count(s->device);
  s->generic_blocks = ce::generic_blocks(S, s->sms);
  s->diag_blocks_max = 8 * s->sms;
  if (cfg->stream) {
    s->stream = static_cast<cudaStream_t>(cfg->stream);
  } else {
    e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete s;
      return cuda_fail(e, "ce_create: stream");
    }
    s->own_stream = true;
  }
  for (int b = 0; b < 2; ++b)
    for (int i = 0; i < s->nf; ++i) {
      s->f[b][i] = dalloc(s, (size_t)S * s->esize);
      s->w[b][i] = dalloc(s, (size_t)S * s->esize);
      if (!s->f[b][i] || !s->w[b][i]) {
        ce_free(s);
        return fail(CE_ENOMEM, "ce_create: device allocation of the lattice state failed");
      }
    }
  if (s->kernel == CE_KERNEL_SWEEP) {
    e = ce::sweep_prepare(s->plan, s->f, s->w, s->N, s->nf, s->prec, s->device, cfg->tile_rows, cfg->stages,
                          cfg->zchunks);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (cfg->kernel == CE_KERNEL_SWEEP) {
        ce_free(s);
        return cuda_fail(e, "ce_create: z-sweep kernel set-up");
      }
      s->kernel = CE_KERNEL_GENERIC;   // e.g. a driver without tensor-map encoding
    }
  }
  // partial sums: room for the largest grid any z-sweep plan can use (8-row tiles, N/2 z-chunks)
  int64_t sweep_blocks = 0;
  if (s->kernel == CE_KERNEL_SWEEP) {
    const int64_t tx = s->prec == CE_F32 ? 128 : 64;
    sweep_blocks = std::max<int64_t>((int64_t)s->plan.gx * s->plan.gy * s->plan.gz, (s->N / tx) * (s->N / 4) * (s->N / 2));
  }
  int64_t planes_blocks = 0;
  if (s->kernel == CE_KERNEL_PLANES && s->dims == 3) {
    s->cols = ce::cols_plan(s->N, s->nf, s->prec, s->sms);
    planes_blocks = (int64_t)s->cols.gx * s->cols.gz;
  } else if (s->kernel == CE_KERNEL_PLANES) {
    s->lines = ce::lines_plan(s->N, s->nf, s->prec, s->sms);
    planes_blocks = (int64_t)s->lines.gx * s->lines.gy;
  }
  int64_t nblk = std::max<int64_t>(std::max<int64_t>(s->generic_blocks, std::max(sweep_blocks, planes_blocks)), 1);
  int64_t plen = std::max<int64_t>(2 * nblk, (int64_t)s->diag_blocks_max * 17);
  s->partials = static_cast<double*>(dalloc(s, (size_t)plen * 8));
  s->aux = static_cast<ce::DevAux*>(dalloc(s, sizeof(ce::DevAux)));
  s->chunk = std::min<int64_t>(S, kStagingChunk);
  s->staging = static_cast<double*>(dalloc(s, (size_t)s->chunk * s->nf * 8));
  if (!s->partials || !s->aux || !s->staging) {
    ce_free(s);
    return fail(CE_ENOMEM, "ce_create: device allocation of scratch failed");
  }
  e = cudaStreamCreateWithFlags(&s->xfer, cudaStreamNonBlocking);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaEventCreateWithFlags(&s->xready[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->xfree[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->xstart, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    ce_free(s);
    return cuda_fail(e, "ce_create: transfer stream");
  }
  if (s->kernel == CE_KERNEL_ROWS) {
    rc = ce::rows_create(s, &s->rows);
    if (rc != CE_OK) {
      if (cfg->kernel == CE_KERNEL_ROWS) {
        ce_free(s);
        return rc;
      }
      cudaGetLastError();
      g_err.clear();
      s->kernel = CE_KERNEL_GENERIC;   // automatic choice: fall back to the generic kernel
    }
  }
  e = cudaMemsetAsync(s->aux, 0, sizeof(ce::DevAux), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    ce_free(s);
    return cuda_fail(e, "ce_create: init");
  }
  *out = s;
  return CE_OK;
}

void ce_free(ce_sim* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  if (s->batch) ce::batch_detach(s->batch, s);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& g : s->graph)
    if (g) cudaGraphExecDestroy(g);
  ce::outputs_release(s);
  ce::rows_free(s->rows);
  if (s->xfer) cudaStreamSynchronize(s->xfer);
  release_all(s);
  if (s->xfer) cudaStreamDestroy(s->xfer);
  for (int b = 0; b < 2; ++b) {
    if (s->xready[b]) cudaEventDestroy(s->xready[b]);
    if (s->xfree[b]) cudaEventDestroy(s->xfree[b]);
  }
  if (s->xstart) cudaEventDestroy(s->xstart);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

int ce_set_fields(ce_sim* s, const double* f, const double* v, int mode, const ce_scalars_t* sc) {
  g_err.clear();
  int rc = check_sim(s, "ce_set_fields");
  if (rc) return rc;
  if (!f || !v) return fail(CE_EINVAL, "ce_set_fields: f and v must be non-NULL");
  if (s->batch) return fail(CE_ESTATE, "ce_set_fields: the handle is a member of a batch (free the batch first)");
  if (mode != CE_VEL_SYNC && mode != CE_VEL_STAGGERED) return fail(CE_EINVAL, "ce_set_fields: unknown mode");
  if (mode == CE_VEL_SYNC && sc) return fail(CE_EINVAL, "ce_set_fields: scalars are only taken with CE_VEL_STAGGERED");
  if (mode == CE_VEL_STAGGERED) {
    if (!sc) return fail(CE_EINVAL, "ce_set_fields: CE_VEL_STAGGERED needs the scalars");
    if (!(sc->a > 0.0) || !std::isfinite(sc->a) || !std::isfinite(sc->ap_half) || !std::isfinite(sc->app) ||
        !std::isfinite(sc->t) || sc->step < 0)
      return fail(CE_EINVAL, "ce_set_fields: scalars must be finite with a > 0 and step >= 0");
  }
  if ((rc = select_device(s))) return rc;
  for (int i = 0; i < s->nf; ++i) {
    if ((rc = upload_field(s, f + (int64_t)i * s->S, s->f[s->cur][i]))) return rc;
    if ((rc = upload_field(s, v + (int64_t)i * s->S, s->w[s->cur][i]))) return rc;
  }
  cudaError_t e = cudaMemsetAsync(&s->aux->status, 0, sizeof(int), s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "ce_set_fields");
  ce::DevAux host{};
  if (mode == CE_VEL_SYNC) {
    // start-up: sums over (f(0), u(0)) -> a'(0), a''(0) -> half kick
    e = run_diag(s, /*raw_u=*/1);
    if (e == cudaSuccess) e = ce::launch_init_scalars(s->aux, s->cur, s->cfg.expansion, s->cfg.dt, s->kappa2, s->stream);
    if (e == cudaSuccess) e = step_once(s, s->cur, /*half_kick=*/true);
    if (e != cudaSuccess) return cuda_fail(e, "ce_set_fields: start-up");
    s->cur ^= 1;
    s->t = 0.0;
    s->step = 0;
  } else {
    ce::DevScalars d{};
    if (s->cfg.expansion) {
      d.a = sc->a;
      d.ap = sc->ap_half;
      d.app = sc->app;
      d.s = sc->app / sc->a;
    } else {
      d.a = 1.0;
    }
    d.c = 0.0;   // the caller's v is f'(t+dt/2) itself
    ce::DevScalars both[2] = {d, d};
    e = cudaMemcpyAsync(s->aux->slot, both, sizeof(both), cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ce_set_fields: scalars");
    s->t = sc->t;
    s->step = sc->step;
  }
  rc = fetch_aux(s, &host);
  if (rc) return rc;
  s->have_state = true;
  return CE_OK;
}

int ce_step(ce_sim* s, int64_t n) {
  g_err.clear();
  int rc = check_sim(s, "ce_step");
  if (rc) return rc;
  if (n < 0) return fail(CE_EINVAL, "ce_step: n must be >= 0");
  if (!s->have_state) return fail(CE_ESTATE, "ce_step: no fields set (call ce_set_fields first)");
  if (s->batch) return fail(CE_ESTATE, "ce_step: the handle is a member of a batch (use ce_batch_step)");
  if ((rc = select_device(s))) return rc;
  while (n >= kGraphSteps && s->graphs_ok) {
    cudaError_t e = ensure_graph(s, s->cur);
    if (e != cudaSuccess) {
      // capture is unavailable on this stream (e.g. the legacy default stream): plain launches
      cudaGetLastError();
      s->graphs_ok = false;
      break;
    }
    e = cudaGraphLaunch(s->graph[s->cur], s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ce_step: graph launch");
    for (int k = 0; k < kGraphSteps; ++k) s->t = s->t + s->cfg.dt;
    s->step += kGraphSteps;
    n -= kGraphSteps;
  }
  for (int64_t k = 0; k < n; ++k) {
    cudaError_t e = step_once(s, s->cur, false);
    if (e != cudaSuccess) return cuda_fail(e, "ce_step: launch");
    s->cur ^= 1;
    s->t = s->t + s->cfg.dt;
    s->step += 1;
  }
  return CE_OK;
}

int ce_synchronize(ce_sim* s) {
  g_err.clear();
  int rc = check_sim(s, "ce_synchronize");
  if (rc) return rc;
  if ((rc = select_device(s))) return rc;
  ce::DevAux host{};
  return fetch_aux(s, &host);
}

int ce_means_variances(ce_sim* s, double* mean, double* var) {
  g_err.clear();
  int rc = check_sim(s, "ce_means_variances");
  if (rc) return rc;
  if (!mean || !var) return fail(CE_EINVAL, "ce_means_variances: NULL output");
  if (!s->have_state) return fail(CE_ESTATE, "ce_means_variances: no fields set");
  if ((rc = select_device(s))) return rc;
  cudaError_t e = run_diag(s, 0);
  if (e != cudaSuccess) return cuda_fail(e, "ce_means_variances");
  ce::DevAux host{};
  if ((rc = fetch_aux(s, &host))) return rc;
  for (int i = 0; i < s->nf; ++i) {
    mean[i] = host.result[ce::R_MEAN + i];
    var[i] = host.result[ce::R_VAR + i];
  }
  return CE_OK;
}

int ce_energy(ce_sim* s, ce_energy_t* out) {
  g_err.clear();
  int rc = check_sim(s, "ce_energy");
  if (rc) return rc;
  if (!out) return fail(CE_EINVAL, "ce_energy: NULL output");
  if (!s->have_state) return fail(CE_ESTATE, "ce_energy: no fields set");
  if ((rc = select_device(s))) return rc;
  cudaError_t e = run_diag(s, 0);
  if (e != cudaSuccess) return cuda_fail(e, "ce_energy");
  ce::DevAux host{};
  if ((rc = fetch_aux(s, &host))) return rc;
  std::memset(out, 0, sizeof(*out));
  for (int i = 0; i < s->nf; ++i) {
    out->K[i] = host.result[ce::R_K + i];
    out->G[i] = host.result[ce::R_G + i];
  }
  out->V = host.result[ce::R_V];
  out->E = host.result[ce::R_E];
  out->a = host.result[ce::R_A];
  out->ap = host.result[ce::R_AP];
  out->friedmann_resid = host.result[ce::R_RESID];
  out->t = s->t;
  out->step = s->step;
  return CE_OK;
}

int ce_get_fields(ce_sim* s, double* f, double* v, int mode, ce_scalars_t* sc) {
  g_err.clear();
  int rc = check_sim(s, "ce_get_fields");
  if (rc) return rc;
  if (!f || !v) return fail(CE_EINVAL, "ce_get_fields: f and v must be non-NULL");
  if (mode != CE_VEL_SYNC && mode != CE_VEL_STAGGERED) return fail(CE_EINVAL, "ce_get_fields: unknown mode");
  if (mode == CE_VEL_STAGGERED && !sc) return fail(CE_EINVAL, "ce_get_fields: CE_VEL_STAGGERED needs sc");
  if (!s->have_state) return fail(CE_ESTATE, "ce_get_fields: no fields set");
  if ((rc = select_device(s))) return rc;
  for (int i = 0; i < s->nf; ++i)
    if ((rc = download_field(s, s->f[s->cur][i], nullptr, f + (int64_t)i * s->S))) return rc;
  if (mode == CE_VEL_STAGGERED) {
    for (int i = 0; i < s->nf; ++i)
      if ((rc = download_field(s, s->f[s->cur][i], s->w[s->cur][i], v + (int64_t)i * s->S))) return rc;
  } else {
    rc = pipelined_download(s, s->nf, v, [&](int64_t s0, int64_t n, double* buf) -> cudaError_t {
      if (s->prec == CE_F32) {
        ce::DiagArgs<float> a = make_diag_args<float>(s, 0);
        a.u_out = buf; a.s0 = s0; a.count = n;
        return ce::launch_sync_u_range<float>(a, s->stream);
      }
      ce::DiagArgs<double> a = make_diag_args<double>(s, 0);
      a.u_out = buf; a.s0 = s0; a.count = n;
      return ce::launch_sync_u_range<double>(a, s->stream);
    }, "ce_get_fields: synchronised velocity");
    if (rc) return rc;
  }
  ce::DevAux host{};
  if ((rc = fetch_aux(s, &host))) return rc;
  if (sc) {
    const ce::DevScalars& d = host.slot[s->cur];
    sc->a = s->cfg.expansion ? d.a : 1.0;
    sc->ap_half = s->cfg.expansion ? d.ap : 0.0;
    sc->app = s->cfg.expansion ? d.app : 0.0;
    sc->t = s->t;
    sc->step = s->step;
  }
  return CE_OK;
}

int64_t ce_device_bytes(const ce_sim* s) { return s ? s->bytes : 0; }

int ce_kernel_in_use(const ce_sim* s) { return s ? s->kernel : CE_KERNEL_GENERIC; }

int ce_replan(ce_sim* s, int rows, int stages, int zchunks) {
  g_err.clear();
  int rc = check_sim(s, "ce_replan");
  if (rc) return rc;
  if (s->batch) return fail(CE_ESTATE, "ce_replan: the handle is a member of a batch");
  if (s->kernel != CE_KERNEL_SWEEP) return fail(CE_EINVAL, "ce_replan: this handle runs the generic kernel");
  if ((rows != 0 && rows != 4 && rows != 8 && rows != 16) || (stages != 0 && (stages < 3 || stages > 5)) || zchunks < 0 ||
      zchunks > s->N / 2 || !ce::sweep_hint_valid(s->N, s->nf, s->prec, rows, stages))
    return fail(CE_EINVAL, "ce_replan: no compiled z-sweep variant matches");
  if ((rc = select_device(s))) return rc;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(e, "ce_replan");
  ce::SweepPlan p{};
  e = ce::sweep_prepare(p, s->f, s->w, s->N, s->nf, s->prec, s->device, rows, stages, zchunks);
  if (e != cudaSuccess) return cuda_fail(e, "ce_replan: plan");
  for (auto& g : s->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  s->graphs_ok = true;
  s->plan = p;
  return CE_OK;
}

int ce_sweep_plan(const ce_sim* s, int* rows, int* stages, int* zchunks) {
  if (!s || !rows || !stages || !zchunks) return fail(CE_EINVAL, "ce_sweep_plan: NULL argument");
  if (s->kernel != CE_KERNEL_SWEEP) {
    *rows = *stages = *zchunks = 0;
    return CE_OK;
  }
  *rows = s->plan.ty;
  *stages = s->plan.stages;
  *zchunks = s->plan.gz;
  return CE_OK;
}

}  // extern "C"
