// Instantiates the templated kernels for one fiber count PRISM_K and exposes them
// through a KernelSet. Included by prism_k<K>.cu.
#include "prism_kernels.cuh"
#include "prism_launch.h"

#ifndef PRISM_K
#error "PRISM_K must be defined"
#endif

namespace prism {
namespace {

constexpr int kK = PRISM_K;

// Launches fn on st, as a programmatic dependent of the stream's previous kernel when `pdl`
// (the kernel then waits for it on the device before reading what it wrote).
template <typename... P, typename... A>
cudaError_t launch_dep(void (*fn)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, bool pdl, A... args) {
  if (!pdl) {
    fn<<<grid, block, smem, st>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, args...);
}

template <int TPV, int LOSS, bool CAL, bool SHELL = false>
cudaError_t fused_one(const IterArgs& a, int grid, int nt, size_t smem, cudaStream_t st) {
  auto fn = k_iter_fused<kK, TPV, LOSS, CAL, SHELL>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  // a programmatic dependent only after k_prior_grad (which lets it start once every one of
  // its CTAs has run past its own wait), and only where the tile queue hands each CTA two tiles
  // or more: CTAs that start early land on the SMs that k_prior_grad leaves free, and with one
  // tile per CTA nothing evens that out (a 40^3 phantom's iteration, 500 tiles on 500 CTAs,
  // took 0.101 instead of 0.075 ms; the brain's, 9.5 tiles per CTA, 0.8 % less time)
  const bool dep = a.pdl && a.nb_priors && a.ntiles >= 2 * grid;
  return launch_dep(fn, dim3(grid), dim3(nt), smem, st, dep, a);
}

template <int TPV, int LOSS, bool CAL, bool SHELL = false>
cudaError_t fused_occ(int nt, size_t smem, int* blocks) {
  auto fn = k_iter_fused<kK, TPV, LOSS, CAL, SHELL>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, fn, nt, smem);
}

template <int TPV>
cudaError_t fused_tpv(const IterArgs& a, int loss, int cal, int grid, int nt, size_t smem, cudaStream_t st) {
  if (loss == kLossMSE) {
    return cal ? fused_one<TPV, kLossMSE, true>(a, grid, nt, smem, st)
               : fused_one<TPV, kLossMSE, false>(a, grid, nt, smem, st);
  }
  return cal ? fused_one<TPV, kLossNLL, true>(a, grid, nt, smem, st)
             : fused_one<TPV, kLossNLL, false>(a, grid, nt, smem, st);
}

template <int TPV>
cudaError_t occ_tpv(int loss, int cal, int nt, size_t smem, int* blocks) {
  if (loss == kLossMSE) {
    return cal ? fused_occ<TPV, kLossMSE, true>(nt, smem, blocks) : fused_occ<TPV, kLossMSE, false>(nt, smem, blocks);
  }
  return cal ? fused_occ<TPV, kLossNLL, true>(nt, smem, blocks) : fused_occ<TPV, kLossNLL, false>(nt, smem, blocks);
}

cudaError_t l_fused(const IterArgs& a, int loss, int cal, int tpv, int shell, int grid, int nt, size_t smem,
                    cudaStream_t st) {
  if constexpr (kK <= 3) {
    if (shell) {
      if (tpv != 1 || loss != kLossMSE || cal) return cudaErrorInvalidValue;
      return fused_one<1, kLossMSE, false, true>(a, grid, nt, smem, st);
    }
  }
  switch (tpv) {
    case 1: return fused_tpv<1>(a, loss, cal, grid, nt, smem, st);
    case 4: return fused_tpv<4>(a, loss, cal, grid, nt, smem, st);
    case 16: return fused_tpv<16>(a, loss, cal, grid, nt, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t l_fused_occupancy(int loss, int cal, int tpv, int shell, int nt, size_t smem, int* blocks) {
  if constexpr (kK <= 3) {
    if (shell) {
      if (tpv != 1 || loss != kLossMSE || cal) return cudaErrorInvalidValue;
      return fused_occ<1, kLossMSE, false, true>(nt, smem, blocks);
    }
  }
  switch (tpv) {
    case 1: return occ_tpv<1>(loss, cal, nt, smem, blocks);
    case 4: return occ_tpv<4>(loss, cal, nt, smem, blocks);
    case 16: return occ_tpv<16>(loss, cal, nt, smem, blocks);
    default: return cudaErrorInvalidValue;
  }
}

inline int nblocks(int64_t n, int b) { return static_cast<int>((n + b - 1) / b); }

cudaError_t l_transform(const IterArgs& a, int tb, int te, cudaStream_t st) {
  const int64_t n = static_cast<int64_t>(te - tb) * a.TV;
  if (n <= 0) return cudaSuccess;
  k_transform<kK><<<nblocks(n, 128), 128, 0, st>>>(a, tb, te);
  return cudaGetLastError();
}

template <int TPV>
cudaError_t synth_tpv(const IterArgs& a, const PlainArgs& p, int cal, int nt, cudaStream_t st) {
  const int g = p.tile_end - p.tile_begin;
  if (cal) k_synth<kK, TPV, true><<<g, nt, 0, st>>>(a, p);
  else k_synth<kK, TPV, false><<<g, nt, 0, st>>>(a, p);
  return cudaGetLastError();
}

cudaError_t l_synth(const IterArgs& a, const PlainArgs& p, int cal, int tpv, int nt, cudaStream_t st) {
  if (p.tile_end <= p.tile_begin) return cudaSuccess;
  switch (tpv) {
    case 1: return synth_tpv<1>(a, p, cal, nt, st);
    case 4: return synth_tpv<4>(a, p, cal, nt, st);
    case 16: return synth_tpv<16>(a, p, cal, nt, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int TPV>
cudaError_t adjoint_tpv(const IterArgs& a, const PlainArgs& p, int cal, int nt, size_t smem, cudaStream_t st) {
  const int g = p.tile_end - p.tile_begin;
  if (cal) {
    auto fn = k_adjoint<kK, TPV, true>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    fn<<<g, nt, smem, st>>>(a, p);
  } else {
    k_adjoint<kK, TPV, false><<<g, nt, 0, st>>>(a, p);
  }
  return cudaGetLastError();
}

cudaError_t l_adjoint(const IterArgs& a, const PlainArgs& p, int cal, int tpv, int nt, size_t smem, cudaStream_t st) {
  if (p.tile_end <= p.tile_begin) return cudaSuccess;
  switch (tpv) {
    case 1: return adjoint_tpv<1>(a, p, cal, nt, smem, st);
    case 4: return adjoint_tpv<4>(a, p, cal, nt, smem, st);
    case 16: return adjoint_tpv<16>(a, p, cal, nt, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t l_prior_prep(const IterArgs& a, int tb, int te, cudaStream_t st) {
  const int64_t n = static_cast<int64_t>(te - tb) * a.TV;
  if (n <= 0) return cudaSuccess;
  return launch_dep(k_prior_prep<kK>, dim3(nblocks(n, 128)), dim3(128), 0, st, a.pdl != 0, a, tb, te);
}

cudaError_t l_prior_grad(const IterArgs& a, int tb, int te, cudaStream_t st) {
  const int64_t n = static_cast<int64_t>(te - tb) * a.TV;
  if (n <= 0) return cudaSuccess;
  return launch_dep(k_prior_grad<kK>, dim3(nblocks(n, 128)), dim3(128), 0, st, a.pdl != 0, a, tb, te);
}

cudaError_t l_prior(const IterArgs& a, const PlainArgs& p, cudaStream_t st) {
  const int g = p.tile_end - p.tile_begin;
  if (g <= 0) return cudaSuccess;
  // one block of TV threads per tile (TV <= 256): the tile's prior value is one block sum
  k_prior<kK><<<dim3(1, g), (a.TV + 31) / 32 * 32, 0, st>>>(a, p);
  return cudaGetLastError();
}

cudaError_t l_fibers(const IterArgs& a, const int32_t* sov, int64_t V, float rel, float* dirs, float* fracs,
                     uint8_t* peaks, cudaStream_t st) {
  if (V <= 0) return cudaSuccess;
  k_fibers<kK><<<nblocks(V, 128), 128, 0, st>>>(a, sov, V, rel, dirs, fracs, peaks);
  return cudaGetLastError();
}
cudaError_t l_stitch(const IterArgs& a, const int32_t* sov, int64_t n_out, const int64_t* src0, const int64_t* src1,
                     const float* w1, float* s0, float* fracs, float* fin, float* dirs, cudaStream_t st) {
  if (n_out <= 0) return cudaSuccess;
  k_stitch<kK><<<nblocks(n_out, 128), 128, 0, st>>>(a, sov, n_out, src0, src1, w1, s0, fracs, fin, dirs);
  return cudaGetLastError();
}

}  // namespace

#define PRISM_CAT2(a, b) a##b
#define PRISM_CAT(a, b) PRISM_CAT2(a, b)
const KernelSet& PRISM_CAT(kernels_k, PRISM_K)() {
  static const KernelSet ks = {l_fused, l_fused_occupancy, l_transform, l_synth, l_adjoint, l_prior_prep, l_prior_grad, l_prior, l_fibers, l_stitch};
  return ks;
}

}  // namespace prism
