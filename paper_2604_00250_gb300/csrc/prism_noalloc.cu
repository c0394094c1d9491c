// Allocation-free evaluation of the voxel-local objective and its gradient.
//
// Who needs it: callers that cannot allocate device memory at the point where they
// evaluate the fit -- code hosted inside a framework that owns the whole device memory
// pool and refuses foreign allocations, real-time pipelines that reserve all memory at
// start-up because cudaMalloc / cudaFree can synchronise the device and stall other
// streams, and plugins whose host forbids allocation outside its own allocator. They
// pass every input and output buffer; the only other memory used is the fixed
// file-scope array below, which every GPU that loads the library holds until exit.
//
// It evaluates, for n_vox voxels of one group, the mean squared error of the predicted
// signal (summed over measurements, divided by n_vox) plus the mean direction-repulsion and
// minor-fraction sparsity penalties (no calibration, no neighbour priors), on raw signal rows
// that it divides by each voxel's mean b <= 50 signal, exactly as prism_forward /
// prism_backward do for such a problem, and writes J and dJ/dtheta. The paper has no
// counterpart of this entry point.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "prism.h"
#include "prism_kernels.cuh"

namespace prism {
namespace {

constexpr int kNaThreads = 128;                        // voxels per block
constexpr int kNaMaxMeas = 1024;                       // table rows
constexpr int kNaMaxBlocks = 8192;                     // loss partials
constexpr int64_t kNaMaxVox = static_cast<int64_t>(kNaMaxBlocks) * kNaThreads;   // 1,048,576
constexpr size_t kNaTableBytes = kNaMaxMeas * sizeof(MeasRow);                   // 64 KiB
constexpr size_t kNaPartialOff = kNaTableBytes;
constexpr size_t kNaCounterOff = kNaPartialOff + kNaMaxBlocks * sizeof(double);  // + 64 KiB
constexpr size_t kNaScratchBytes = kNaCounterOff + 256;

// The scratch: measurement table, per-block loss partials, arrival counter. Shared by
// every call on a device; the last call's contents stay until the next call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

// Host side: the array's device address, looked up once per device.
std::mutex g_na_mutex;
void* g_na_addr[64] = {};

template <int K>
__global__ void __launch_bounds__(kNaThreads) k_grad_noalloc(const float* __restrict__ signal,
                                                            const float* __restrict__ theta, int64_t V, int N,
                                                            float lam_rep, float lam_sparse, float tau,
                                                            float* __restrict__ grad, double* __restrict__ loss,
                                                            unsigned char* scratch) {
  constexpr int NF = K + 3, Q = 4 * K + 5;
  extern __shared__ __align__(16) MeasRow s_tab[];
  __shared__ double s_red[8][3];
  __shared__ int s_last;
  const MeasRow* tab = reinterpret_cast<const MeasRow*>(scratch);
  double* partial = reinterpret_cast<double*>(scratch + kNaPartialOff);
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNaCounterOff);
  for (int n = threadIdx.x; n < N; n += blockDim.x) s_tab[n] = tab[n];
  __syncthreads();
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool act = v < V;
  const float inv_M = 1.f / static_cast<float>(V);
  float th[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) th[q] = act ? theta[v * Q + q] : 0.f;
  Vox<K> P;
  transform<K>(th, P);
  float ffin[K], fomf[K];
  fiber_weights<K>(P, ffin, fomf);
  // b0 normalisation: mean of the b <= 50 measurements, table rows flagged by pad0. A mean
  // that is not positive and finite is replaced by 1 for this voxel's arithmetic (as the
  // handle path's b0 statistics do) and marks the voxel: its gradient row and the loss
  // become NaN, since an asynchronous call cannot return an error code for it.
  float b0 = 1.f;
  bool bad = false;
  if (act) {
    double m = 0.0;
    int nb0 = 0;
    for (int n = 0; n < N; ++n)
      if (s_tab[n].pad0 != 0.f) {
        m += signal[v * N + n];
        ++nb0;
      }
    const double mean = m / nb0;
    if (mean > 0.0 && mean < 1e300) {
      b0 = static_cast<float>(mean);
    } else {
      bad = true;
    }
  }
  Acc<K> A;
  acc_zero<K>(A);
  if (act) {
    for (int n = 0; n < N; ++n) {
      float rr, u;
      pair<K, kLossMSE, false, false>(P, ffin, fomf, s_tab[n], signal[v * N + n] / b0, 1.f, 0.f, 0.f, A, rr, u);
    }
  }
  float gS0, gf[NF], gd[K][3], gfin;
  data_grad<K>(P, A, 2.f * inv_M, gS0, gf, gd, gfin);
  IterArgs pa{};
  pa.lam_rep = lam_rep;
  pa.lam_sparse = lam_sparse;
  pa.tau = tau;
  pa.nb_priors = 0;
  const float ploss = act ? priors<K>(pa, P, 0, inv_M, nullptr, gS0, gf, gd) : 0.f;
  float g[Q];
  chain_raw<K>(P, gS0, gf, gd, gfin, g);
  const float qnan = __int_as_float(0x7fc00000);
  if (act) {
#pragma unroll
    for (int q = 0; q < Q; ++q) grad[v * Q + q] = bad ? qnan : g[q];
  }
  double out[3];
  const double dl = bad ? static_cast<double>(qnan) : static_cast<double>(A.l1 * inv_M);
  block_reduce3(act ? dl : 0.0, act ? static_cast<double>(ploss) : 0.0, 0.0, s_red, out);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = out[0] + out[1];
    __threadfence();
    s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    double tot = 0.0;
    for (unsigned int b = 0; b < gridDim.x; ++b) tot += __ldcg(&partial[b]);
    *loss = tot;
    *counter = 0u;
  }
}

}  // namespace
}  // namespace prism

using namespace prism;

// Defined in prism_api.cu: records the message returned by prism_last_error().
int prism_record_error(int code, const char* msg);

extern "C" int prism_grad_noalloc(const float* signal, const float* bvals, const float* bvecs, const float* theta,
                                  int64_t n_vox, int32_t n_meas, int32_t K, float lam_rep, float lam_sparse,
                                  float tau, float* grad, double* loss, void* stream) {
  if (!signal || !bvals || !bvecs || !theta || !grad || !loss)
    return prism_record_error(PRISM_E_INVALID_ARG, "prism_grad_noalloc: NULL argument");
  if (K < 1 || K > PRISM_MAX_K) return prism_record_error(PRISM_E_INVALID_ARG, "prism_grad_noalloc: K must be in 1..5");
  if (n_vox < 1 || n_vox > kNaMaxVox)
    return prism_record_error(PRISM_E_SHAPE, ("prism_grad_noalloc: n_vox must be in 1.." + std::to_string(kNaMaxVox) +
                                              " (the fixed scratch holds " + std::to_string(kNaMaxBlocks) +
                                              " block partials of 128 voxels)").c_str());
  if (n_meas < 1 || n_meas > kNaMaxMeas)
    return prism_record_error(PRISM_E_SHAPE, "prism_grad_noalloc: n_meas must be in 1..1024");
  if (!(lam_rep >= 0.f) || !(lam_sparse >= 0.f) || !(tau >= 0.f))
    return prism_record_error(PRISM_E_INVALID_ARG, "prism_grad_noalloc: lam_rep, lam_sparse and tau must be >= 0");
  // measurement table on the host (float copies of double constants), b=0 rows flagged
  static thread_local MeasRow rows[kNaMaxMeas];
  int nb0 = 0;
  const double L2E = 1.4426950408889634, dpar = 1.7e-3, dperp = 0.4e-3;
  for (int n = 0; n < n_meas; ++n) {
    const double b = bvals[n];
    if (!std::isfinite(b) || b < 0.0) return prism_record_error(PRISM_E_INVALID_ARG, "prism_grad_noalloc: bad b-value");
    // the b-vector rules of prism_fit_init: finite, and unit length where b > 50
    const float gx = bvecs[3 * n], gy = bvecs[3 * n + 1], gz = bvecs[3 * n + 2];
    if (!std::isfinite(gx) || !std::isfinite(gy) || !std::isfinite(gz))
      return prism_record_error(PRISM_E_INVALID_ARG, "prism_grad_noalloc: non-finite b-vector");
    if (b > 50.0 && std::fabs(std::sqrt(gx * gx + gy * gy + gz * gz) - 1.f) > 1e-3f)
      return prism_record_error(PRISM_E_INVALID_ARG,
                                ("prism_grad_noalloc: b-vector " + std::to_string(n) +
                                 " of a b > 50 measurement is not unit length").c_str());
    MeasRow r;
    r.gx = bvecs[3 * n];
    r.gy = bvecs[3 * n + 1];
    r.gz = bvecs[3 * n + 2];
    r.nkpar = static_cast<float>(-b * dpar * L2E);
    r.nkperp = static_cast<float>(-b * dperp * L2E);
    r.nkd = static_cast<float>(-b * (dpar - dperp) * L2E);
    r.ecsf = static_cast<float>(std::exp(-b * 3.0e-3));
    r.egm = static_cast<float>(std::exp(-b * 0.9e-3));
    r.eres = static_cast<float>(std::exp(-b * 0.2e-3));
    r.An = static_cast<float>(-2.0 * b * dpar);
    r.Bn = static_cast<float>(2.0 * b * (dperp - dpar));
    r.A = 1.f;
    r.beta = 0.f;
    r.pad0 = (b <= 50.0) ? 1.f : 0.f;
    r.pad1 = r.pad2 = 0.f;
    nb0 += (b <= 50.0);
    rows[n] = r;
  }
  if (nb0 == 0) return prism_record_error(PRISM_E_SHAPE, "prism_grad_noalloc: no b <= 50 measurement");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64)
    return prism_record_error(PRISM_E_CUDA, "prism_grad_noalloc: cudaGetDevice failed");
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return prism_record_error(PRISM_E_CUDA, (std::string("prism_grad_noalloc: cudaGetSymbolAddress: ") +
                                                 cudaGetErrorString(e)).c_str());
      g_na_addr[dev] = p;
    }
    scratch = static_cast<unsigned char*>(g_na_addr[dev]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  e = cudaMemsetAsync(scratch + kNaCounterOff, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(scratch, rows, n_meas * sizeof(MeasRow), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess)
    return prism_record_error(PRISM_E_CUDA, (std::string("prism_grad_noalloc: ") + cudaGetErrorString(e)).c_str());
  const int blocks = static_cast<int>((n_vox + kNaThreads - 1) / kNaThreads);
  const size_t smem = static_cast<size_t>(n_meas) * sizeof(MeasRow);
  auto go = [&](auto fn) {
    cudaError_t r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (r != cudaSuccess) return r;
    fn<<<blocks, kNaThreads, smem, st>>>(signal, theta, n_vox, n_meas, lam_rep, lam_sparse, tau, grad, loss, scratch);
    return cudaGetLastError();
  };
  switch (K) {
    case 1: e = go(k_grad_noalloc<1>); break;
    case 2: e = go(k_grad_noalloc<2>); break;
    case 3: e = go(k_grad_noalloc<3>); break;
    case 4: e = go(k_grad_noalloc<4>); break;
    default: e = go(k_grad_noalloc<5>); break;
  }
  if (e != cudaSuccess)
    return prism_record_error(PRISM_E_CUDA, (std::string("prism_grad_noalloc launch: ") + cudaGetErrorString(e)).c_str());
  return PRISM_OK;
}
