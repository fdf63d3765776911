// ce_outputs.cu -- outputs beyond the means and energies: the binned power
// spectrum of a field (cuFFT transform + binning kernel), the grid-image file
// (a complete state that ce_load restores exactly; arXiv:0712.0813 Sec. II
// describes grid images that let a run be resumed later), and the state at
// chosen sites (a gather, for probing lattices too large to download).
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ce_device.cuh"
#include "ce_internal.h"
#include "clusterlat.h"

namespace {

int ofail(int code, const std::string& msg) {
  ce::set_last_error(msg);
  return code;
}

int ocuda(cudaError_t e, const char* what) {
  ce::set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
  return CE_ECUDA;
}

// f(t) and f'(t + dt/2) = w + c f at m chosen sites, for every field; the
// velocity is rounded in T exactly as the step kernels and ce_get_fields form it.
template <typename T>
struct SamplePtrs {
  const T* f[4];
  const T* w[4];
};

template <typename T>
__global__ void k_sample(SamplePtrs<T> p, int nf, const ce::DevScalars* sc, const int64_t* __restrict__ sites,
                         int64_t m, double* __restrict__ out_f, double* __restrict__ out_v) {
  const T c = (T)sc->c;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = sites[k];
    for (int i = 0; i < nf; ++i) {
      const T fv = p.f[i][x], wv = p.w[i][x];
      out_f[(int64_t)i * m + k] = (double)fv;
      out_v[(int64_t)i * m + k] = (double)ce::fmaT(c, fv, wv);
    }
  }
}

constexpr int kBinThreads = 256;
constexpr int kBinBlocks = 608;

// Signed integer mode of index i along an axis of length N.
__device__ __forceinline__ int64_t mode(int64_t i, int64_t N) { return i <= N / 2 ? i : i - N; }

// Half-spectrum layout of a real-to-complex transform: the last (x) axis holds
// N/2 + 1 modes.  Every stored mode except kx = 0 and the Nyquist kx = N/2
// stands for itself and its complex conjugate at -n, so it counts twice.
// The transform is taken of f - f(site 0), which keeps the large mean of phi
// out of the FFT's rounding; the zero mode gets S f(site 0) back in FP64.
template <typename T>
__global__ void k_shifted_copy(const T* __restrict__ f, T* __restrict__ out, int64_t n) {
  const T shift = f[0];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = f[k] - shift;
}

template <typename C, typename T>
__global__ void __launch_bounds__(kBinThreads) k_bin_spectrum(const C* __restrict__ F, const T* __restrict__ f,
                                                               int64_t N, int dims, int nbins,
                                                               double* __restrict__ part_p,
                                                               double* __restrict__ part_n) {
  extern __shared__ double sh[];
  double* hp = sh;
  double* hn = sh + nbins;
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    hp[b] = 0.0;
    hn[b] = 0.0;
  }
  __syncthreads();
  const int64_t nx = N / 2 + 1;
  int64_t total = nx;
  for (int d = 1; d < dims; ++d) total *= N;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ix = k % nx;
    int64_t rest = k / nx;
    double n2 = (double)ix * (double)ix;
    for (int d = 1; d < dims; ++d) {
      const int64_t m = mode(rest % N, N);
      rest /= N;
      n2 += (double)m * (double)m;
    }
    const int b = (int)floor(sqrt(n2) + 0.5);
    if (b >= nbins) continue;
    const double w = (ix == 0 || (N % 2 == 0 && ix == N / 2)) ? 1.0 : 2.0;
    double re = (double)F[k].x;
    const double im = (double)F[k].y;
    if (k == 0) re += (double)f[0] * (double)(total / nx * N);  // S f(site 0)
    atomicAdd(&hp[b], w * (re * re + im * im));
    atomicAdd(&hn[b], w);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    part_p[(int64_t)blockIdx.x * nbins + b] = hp[b];
    part_n[(int64_t)blockIdx.x * nbins + b] = hn[b];
  }
}

__global__ void k_spectrum_finalize(const double* __restrict__ part_p, const double* __restrict__ part_n, int blocks,
                                    int nbins, double* __restrict__ p_out, double* __restrict__ n_out) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
    double p = 0.0, n = 0.0;
    for (int k = 0; k < blocks; ++k) {  // fixed order over blocks
      p += part_p[(int64_t)k * nbins + b];
      n += part_n[(int64_t)k * nbins + b];
    }
    p_out[b] = n > 0.0 ? p / n : 0.0;
    n_out[b] = n;
  }
}

struct SpectrumWork {
  cufftHandle plan = 0;
  bool have_plan = false;
  void* spec = nullptr;      // complex half spectrum
  void* real = nullptr;      // f - f(site 0), the transform's input
  double* part = nullptr;    // per-block histograms (2 x blocks x nbins_max)
  double* out = nullptr;     // 2 x nbins_max
  int nbins_max = 0;
};

std::vector<std::pair<const ce_sim*, SpectrumWork>>& work_table() {
  static std::vector<std::pair<const ce_sim*, SpectrumWork>> t;
  return t;
}

SpectrumWork* find_work(const ce_sim* s, bool create) {
  for (auto& e : work_table())
    if (e.first == s) return &e.second;
  if (!create) return nullptr;
  work_table().push_back({s, SpectrumWork{}});
  return &work_table().back().second;
}

constexpr char kMagic[8] = {'C', 'E', 'G', 'R', 'I', 'D', '0', '1'};

struct FileHeader {
  char magic[8];
  int32_t dims, nfields, precision, expansion;
  int64_t N;
  double L, dt, q[3], kappa2;
  double a, ap_half, app, t;
  int64_t step;
};

}  // namespace

// Release the spectrum work buffers of a handle (called from ce_free).
void ce::outputs_release(const ce_sim* s) {
  auto& t = work_table();
  for (size_t i = 0; i < t.size(); ++i) {
    if (t[i].first != s) continue;
    SpectrumWork& w = t[i].second;
    if (w.have_plan) cufftDestroy(w.plan);
    if (w.spec) cudaFree(w.spec);
    if (w.real) cudaFree(w.real);
    if (w.part) cudaFree(w.part);
    if (w.out) cudaFree(w.out);
    t.erase(t.begin() + (long)i);
    return;
  }
}

extern "C" {

int ce_spectrum(ce_sim* s, int field, int nbins, double* k, double* power, double* count) {
  ce::set_last_error("");
  if (!s) return ofail(CE_EINVAL, "ce_spectrum: sim is NULL");
  if (!k || !power || !count) return ofail(CE_EINVAL, "ce_spectrum: NULL output");
  if (field < 0 || field >= s->nf) return ofail(CE_EINVAL, "ce_spectrum: field out of range");
  if (!s->have_state) return ofail(CE_ESTATE, "ce_spectrum: no fields set");
  const int max_bins = (int)std::ceil(std::sqrt((double)s->dims) * (double)(s->N / 2)) + 2;
  if (nbins < 1 || nbins > max_bins)
    return ofail(CE_EINVAL, "ce_spectrum: nbins must be 1..ceil(sqrt(dims) N/2) + 2");
  cudaError_t e = cudaSetDevice(s->device);
  if (e == cudaSuccess && s->batch) e = ce::batch_wait(s->batch);
  if (e != cudaSuccess) return ocuda(e, "ce_spectrum");
  SpectrumWork* w = find_work(s, true);
  const bool f32 = s->prec == CE_F32;
  int64_t half = s->N / 2 + 1;
  for (int d = 1; d < s->dims; ++d) half *= s->N;
  if (!w->have_plan) {
    int n[3] = {(int)s->N, (int)s->N, (int)s->N};
    cufftResult r = cufftPlanMany(&w->plan, s->dims, n, nullptr, 1, 0, nullptr, 1, 0, f32 ? CUFFT_R2C : CUFFT_D2Z, 1);
    if (r != CUFFT_SUCCESS) return ofail(CE_ECUDA, "ce_spectrum: cufft plan failed");
    w->have_plan = true;
    e = cudaMalloc(&w->spec, (size_t)half * (f32 ? sizeof(cufftComplex) : sizeof(cufftDoubleComplex)));
    if (e == cudaSuccess) e = cudaMalloc(&w->real, (size_t)s->S * s->esize);
    if (e == cudaSuccess) e = cudaMalloc(&w->part, sizeof(double) * 2 * kBinBlocks * max_bins);
    if (e == cudaSuccess) e = cudaMalloc(&w->out, sizeof(double) * 2 * max_bins);
    if (e != cudaSuccess) {
      ce::outputs_release(s);
      return ofail(CE_ENOMEM, "ce_spectrum: work buffers");
    }
    w->nbins_max = max_bins;
  }
  cufftSetStream(w->plan, s->stream);
  const int cblocks = (int)std::min<int64_t>((s->S + 255) / 256, (int64_t)s->sms * 8);
  if (f32)
    k_shifted_copy<float><<<cblocks, 256, 0, s->stream>>>(static_cast<const float*>(s->f[s->cur][field]),
                                                           static_cast<float*>(w->real), s->S);
  else
    k_shifted_copy<double><<<cblocks, 256, 0, s->stream>>>(static_cast<const double*>(s->f[s->cur][field]),
                                                            static_cast<double*>(w->real), s->S);
  e = cudaGetLastError();
  if (e != cudaSuccess) return ocuda(e, "ce_spectrum: shift");
  cufftResult r;
  if (f32)
    r = cufftExecR2C(w->plan, static_cast<cufftReal*>(w->real), static_cast<cufftComplex*>(w->spec));
  else
    r = cufftExecD2Z(w->plan, static_cast<cufftDoubleReal*>(w->real), static_cast<cufftDoubleComplex*>(w->spec));
  if (r != CUFFT_SUCCESS) return ofail(CE_ECUDA, "ce_spectrum: cufft exec failed");
  double* part_p = w->part;
  double* part_n = w->part + (int64_t)kBinBlocks * nbins;
  const size_t shm = sizeof(double) * 2 * nbins;
  if (f32)
    k_bin_spectrum<cufftComplex, float><<<kBinBlocks, kBinThreads, shm, s->stream>>>(
        static_cast<const cufftComplex*>(w->spec), static_cast<const float*>(s->f[s->cur][field]), s->N, s->dims,
        nbins, part_p, part_n);
  else
    k_bin_spectrum<cufftDoubleComplex, double><<<kBinBlocks, kBinThreads, shm, s->stream>>>(
        static_cast<const cufftDoubleComplex*>(w->spec), static_cast<const double*>(s->f[s->cur][field]), s->N,
        s->dims, nbins, part_p, part_n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return ocuda(e, "ce_spectrum: binning");
  k_spectrum_finalize<<<(nbins + 127) / 128, 128, 0, s->stream>>>(part_p, part_n, kBinBlocks, nbins, w->out,
                                                                   w->out + nbins);
  std::vector<double> host(2 * (size_t)nbins);
  e = cudaMemcpyAsync(host.data(), w->out, sizeof(double) * 2 * nbins, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return ocuda(e, "ce_spectrum: read-back");
  const double two_pi_over_L = 2.0 * M_PI / s->cfg.L;
  for (int b = 0; b < nbins; ++b) {
    k[b] = two_pi_over_L * b;
    power[b] = host[b];
    count[b] = host[nbins + b];
  }
  return CE_OK;
}

int ce_sample_fields(ce_sim* s, const int64_t* sites, int64_t n, double* f, double* v, ce_scalars_t* sc) {
  ce::set_last_error("");
  if (!s) return ofail(CE_EINVAL, "ce_sample_fields: sim is NULL");
  if (n < 0 || (n > 0 && (!sites || !f || !v)) || !sc) return ofail(CE_EINVAL, "ce_sample_fields: bad arguments");
  if (!s->have_state) return ofail(CE_ESTATE, "ce_sample_fields: no fields set");
  for (int64_t k = 0; k < n; ++k)
    if (sites[k] < 0 || sites[k] >= s->S) return ofail(CE_EINVAL, "ce_sample_fields: site index out of range");
  cudaError_t e = cudaSetDevice(s->device);
  if (e == cudaSuccess && s->batch) e = ce::batch_wait(s->batch);
  if (e != cudaSuccess) return ocuda(e, "ce_sample_fields");
  // the staging buffer (chunk x nf doubles) holds, per pass, m site indices and
  // the m x nf values of f and of v
  const int64_t cap = s->chunk * s->nf * 8;
  const int64_t mmax = std::max<int64_t>(1, cap / (8 + 16 * (int64_t)s->nf));
  unsigned char* stage = reinterpret_cast<unsigned char*>(s->staging);
  const void* slot = &s->aux->slot[s->cur];
  for (int64_t k0 = 0; k0 < n; k0 += mmax) {
    const int64_t m = std::min<int64_t>(mmax, n - k0);
    int64_t* d_sites = reinterpret_cast<int64_t*>(stage);
    double* d_f = reinterpret_cast<double*>(stage + m * 8);
    double* d_v = d_f + m * s->nf;
    e = cudaMemcpyAsync(d_sites, sites + k0, (size_t)m * 8, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return ocuda(e, "ce_sample_fields: site upload");
    const int blocks = (int)std::min<int64_t>((m + 255) / 256, (int64_t)s->sms * 4);
    if (s->prec == CE_F32) {
      SamplePtrs<float> p{};
      for (int i = 0; i < s->nf; ++i) {
        p.f[i] = static_cast<const float*>(s->f[s->cur][i]);
        p.w[i] = static_cast<const float*>(s->w[s->cur][i]);
      }
      k_sample<float><<<blocks, 256, 0, s->stream>>>(p, s->nf, static_cast<const ce::DevScalars*>(slot), d_sites, m,
                                                     d_f, d_v);
    } else {
      SamplePtrs<double> p{};
      for (int i = 0; i < s->nf; ++i) {
        p.f[i] = static_cast<const double*>(s->f[s->cur][i]);
        p.w[i] = static_cast<const double*>(s->w[s->cur][i]);
      }
      k_sample<double><<<blocks, 256, 0, s->stream>>>(p, s->nf, static_cast<const ce::DevScalars*>(slot), d_sites, m,
                                                      d_f, d_v);
    }
    e = cudaGetLastError();
    for (int i = 0; i < s->nf && e == cudaSuccess; ++i) {
      e = cudaMemcpyAsync(f + (int64_t)i * n + k0, d_f + (int64_t)i * m, (size_t)m * 8, cudaMemcpyDeviceToHost,
                          s->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(v + (int64_t)i * n + k0, d_v + (int64_t)i * m, (size_t)m * 8, cudaMemcpyDeviceToHost,
                            s->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return ocuda(e, "ce_sample_fields: gather");
  }
  ce::DevAux host{};
  e = cudaMemcpyAsync(&host, s->aux, sizeof(host), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return ocuda(e, "ce_sample_fields: scalars");
  if (host.status != CE_OK) return ofail(host.status, "ce_sample_fields: the device reported an error");
  const ce::DevScalars& d = host.slot[s->cur];
  sc->a = s->cfg.expansion ? d.a : 1.0;
  sc->ap_half = s->cfg.expansion ? d.ap : 0.0;
  sc->app = s->cfg.expansion ? d.app : 0.0;
  sc->t = s->t;
  sc->step = s->step;
  return CE_OK;
}

int ce_save(ce_sim* s, const char* path) {
  ce::set_last_error("");
  if (!s || !path) return ofail(CE_EINVAL, "ce_save: NULL argument");
  if (!s->have_state) return ofail(CE_ESTATE, "ce_save: no fields set");
  const size_t n = (size_t)s->nf * (size_t)s->S;
  std::vector<double> f(n), v(n);
  ce_scalars_t sc;
  int rc = ce_get_fields(s, f.data(), v.data(), CE_VEL_STAGGERED, &sc);
  if (rc != CE_OK) return rc;
  FileHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.dims = s->dims;
  h.nfields = s->nf;
  h.precision = s->prec;
  h.expansion = s->cfg.expansion;
  h.N = s->N;
  h.L = s->cfg.L;
  h.dt = s->cfg.dt;
  for (int i = 0; i < 3; ++i) h.q[i] = s->cfg.q[i];
  h.kappa2 = s->kappa2;
  h.a = sc.a;
  h.ap_half = sc.ap_half;
  h.app = sc.app;
  h.t = sc.t;
  h.step = sc.step;
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return ofail(CE_EINVAL, std::string("ce_save: cannot open ") + path);
  bool ok = std::fwrite(&h, sizeof(h), 1, fp) == 1 && std::fwrite(f.data(), sizeof(double), n, fp) == n &&
            std::fwrite(v.data(), sizeof(double), n, fp) == n;
  ok = (std::fclose(fp) == 0) && ok;
  return ok ? CE_OK : ofail(CE_EINVAL, std::string("ce_save: write failed for ") + path);
}

int ce_load(ce_sim* s, const char* path) {
  ce::set_last_error("");
  if (!s || !path) return ofail(CE_EINVAL, "ce_load: NULL argument");
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return ofail(CE_EINVAL, std::string("ce_load: cannot open ") + path);
  FileHeader h;
  if (std::fread(&h, sizeof(h), 1, fp) != 1 || std::memcmp(h.magic, kMagic, 8) != 0) {
    std::fclose(fp);
    return ofail(CE_EINVAL, "ce_load: not a grid image");
  }
  if (h.dims != s->dims || h.N != s->N || h.nfields != s->nf || h.expansion != s->cfg.expansion ||
      h.L != s->cfg.L || h.dt != s->cfg.dt || h.q[0] != s->cfg.q[0] || h.q[1] != s->cfg.q[1] ||
      h.q[2] != s->cfg.q[2] || h.kappa2 != s->kappa2) {
    std::fclose(fp);
    return ofail(CE_EINVAL, "ce_load: the image was written for another lattice or model");
  }
  const size_t n = (size_t)s->nf * (size_t)s->S;
  std::vector<double> f(n), v(n);
  const bool ok = std::fread(f.data(), sizeof(double), n, fp) == n && std::fread(v.data(), sizeof(double), n, fp) == n;
  std::fclose(fp);
  if (!ok) return ofail(CE_EINVAL, "ce_load: truncated image");
  ce_scalars_t sc{h.a, h.ap_half, h.app, h.t, h.step};
  return ce_set_fields(s, f.data(), v.data(), CE_VEL_STAGGERED, &sc);
}

}  // extern "C"
