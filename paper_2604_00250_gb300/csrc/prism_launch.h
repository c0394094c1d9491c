// Host-side launch interface between the C-ABI implementation and the kernels.
#pragma once

#include <cuda_runtime.h>

#include "prism_device.cuh"

namespace prism {

// Per-K launchers of the templated kernels (one translation unit per K).
struct KernelSet {
  // shell = 1: the shell loop of one thread per voxel, MSE, no calibration (K <= 3)
  cudaError_t (*fused)(const IterArgs& a, int loss, int cal, int tpv, int shell, int grid, int nt, size_t smem,
                       cudaStream_t st);
  cudaError_t (*fused_occupancy)(int loss, int cal, int tpv, int shell, int nt, size_t smem, int* blocks);
  cudaError_t (*transform)(const IterArgs& a, int tb, int te, cudaStream_t st);
  cudaError_t (*synth)(const IterArgs& a, const PlainArgs& p, int cal, int tpv, int nt, cudaStream_t st);
  cudaError_t (*adjoint)(const IterArgs& a, const PlainArgs& p, int cal, int tpv, int nt, size_t smem,
                         cudaStream_t st);
  cudaError_t (*prior_prep)(const IterArgs& a, int tb, int te, cudaStream_t st);
  cudaError_t (*prior_grad)(const IterArgs& a, int tb, int te, cudaStream_t st);
  cudaError_t (*prior)(const IterArgs& a, const PlainArgs& p, cudaStream_t st);
  cudaError_t (*fibers)(const IterArgs& a, const int32_t* slot_of_vox, int64_t V, float rel, float* dirs,
                        float* fracs, uint8_t* peaks, cudaStream_t st);
  cudaError_t (*stitch)(const IterArgs& a, const int32_t* slot_of_vox, int64_t n_out, const int64_t* src0,
                        const int64_t* src1, const float* w1, float* s0, float* fracs, float* fin, float* dirs,
                        cudaStream_t st);
};

const KernelSet& kernels_for_k(int K);

// Group-level kernels (prism_aux.cu).
struct GroupArgs {
  int32_t G, max_split, split_tiles, max_e;
  const int32_t* split_off;   // [G] first part2 row of the group
  double* part2;              // [sum splits][max_e]
  int32_t* counters;          // [G][ceil(max_e / 256)]
  double* gred;               // packed like gparams (double); loss kept separately
  double* gloss;              // [G] data term, then the full objective after finalisation
  double* gprior;             // [G] prior total
  float* gm;                  // group Adam moments (packed like gparams)
  float* gv;
  float* gparams;
  MeasRow* table;
  MeasPair* table2;   // the paired copy (its e^alpha_n and beta_n follow the rows)
  const int32_t* slot_of_grid;
  double* hist;               // [H][G] loss history
  int32_t hist_len;
  float* gexport;             // packed group gradients for the caller (or null)
  int32_t loss_mode;          // kLossMSE / kLossNLL
  float w_alpha, w_beta, w_blr;
  double* bscratch;           // bias-gradient partial contractions (see k_bias_grad_*)
  const int64_t* bs_off;      // [G][2] offsets of a group's [nx][ny][8] and [nx][8][8] parts
  int32_t max_nx, max_ny;     // largest grid extents over the groups
  int32_t* gdone;             // blocks of k_group_adam that finished (last one resets it)
};

cudaError_t launch_group_reduce(const IterArgs& a, const GroupArgs& g, int what, cudaStream_t st);
cudaError_t launch_bias_grad(const IterArgs& a, const GroupArgs& g, cudaStream_t st);
cudaError_t launch_group_adam(const IterArgs& a, const GroupArgs& g, int mode, cudaStream_t st);
cudaError_t launch_loss(const IterArgs& a, const PlainArgs& p, int loss, cudaStream_t st);
cudaError_t launch_adam_voxel(const IterArgs& a, const PlainArgs& p, cudaStream_t st);

// Preprocessing and layout kernels.
cudaError_t launch_b0_stats(const float* sig, int64_t V, int N, const uint8_t* isb0, int nb0,
                            float* b0mean, double* part, int* bad, cudaStream_t st);
cudaError_t launch_sigma_init(const double* part, int nblocks, int64_t V, int nb0, float sigma_fallback,
                              float* sigma_log_out, cudaStream_t st);
cudaError_t launch_pack(const IterArgs& a, const float* sig, const float* b0mean, const int32_t* vox_of_slot,
                        const int32_t* order, int64_t vox0, int tile_begin, int tile_end, int N, float* ypack,
                        int* bad, cudaStream_t st);
cudaError_t launch_slot_data(const Tile* tiles, const GroupDev* groups, int G, const GroupDev* host_groups,
                             const int32_t* slot_of_grid, const int32_t* slot_of_vox, int64_t V, int Vp, int TV, int nnb,
                             int32_t* vox_of_slot, uint32_t* vcoord, uint32_t* vflag, int32_t* nbr, cudaStream_t st);
cudaError_t launch_gather_rows(const float* src, const int64_t* rows, int64_t n, int len, float* dst,
                               cudaStream_t st);
cudaError_t launch_table(const float* bvals, const float* bvecs, int N, MeasRow* rows, cudaStream_t st);
cudaError_t launch_pair_table(const MeasRow* rows, int N, MeasPair* out, cudaStream_t st);
cudaError_t launch_scatter_params(const float* in, const int32_t* slot_of_vox, int64_t V, int Q, int Vpad,
                                  float* theta, cudaStream_t st);
cudaError_t launch_gather_params(const float* theta, const int32_t* slot_of_vox, int64_t V, int Q, int Vpad,
                                 float* out, cudaStream_t st);
cudaError_t launch_default_init(const int32_t* slot_of_vox, const uint32_t* vcoord, int ny, int nz, int64_t V, int K,
                                int Vpad, uint64_t seed, float* theta, cudaStream_t st);
cudaError_t launch_gather_yhat(const float* ypack, const IterArgs& a, const int32_t* vox_of_slot,
                               const int64_t* yhat_row_off, const int32_t* order, float* out, cudaStream_t st);
cudaError_t launch_table_refresh(const GroupArgs& g, const IterArgs& a, cudaStream_t st);
cudaError_t launch_adam_constants(const IterArgs& a, cudaStream_t st);
cudaError_t launch_wait_probe(int32_t* status, int polls, cudaStream_t st);

}  // namespace prism
