/*
 * prism.h -- C-ABI of the GB300 (sm_103a) PRISM fitting library.
 *
 * PRISM (Abouagour, Shah, Garyfallidis, "PRISM: Differentiable Analysis-by-
 * Synthesis for Fixel Recovery in Diffusion MRI") fits, per voxel x of a brain
 * mask and measurement n (b-value b_n, unit gradient g_n), the forward model
 *
 *   S(x,n)    = S0 (f_csf E_csf + f_gm E_gm + sum_k f_wm,k E_wm,k + f_res E_res)   Sec. 2.2, Eq. 3
 *   E_iso     = exp(-b D_iso), D = 3.0 / 0.9 / 0.2 x 1e-3 mm^2/s                   Sec. 2.2, Eq. 4
 *   E_wm,k    = f_in e^{-b D_par c^2} + (1-f_in) e^{-b (D_par c^2 + D_perp (1-c^2))},
 *               c = d_k . g_n, D_par = 1.7e-3, D_perp = 0.4e-3                     Sec. 2.2, Eq. 5
 *   y_hat     = exp(alpha_n) B(x) S(x,n) + beta_n, B = exp(trilinear(b_lr 8^3))    Sec. 2.3, Eq. 6
 *
 * to b0-normalised data y (Sec. 2.5) by minimising the MSE (Eq. 8) or the
 * Rician NLL with learned sigma = exp(sigma_log) (Eq. 9), plus the priors of
 * Sec. 2.4, with Adam (the Table 2 comparator). Each iteration computes the
 * objective, its exact gradient (hand-written adjoint) and one Adam update of
 * every parameter.
 *
 * Conventions
 *  - Every function returns PRISM_OK (0) or a prism_status code; the message
 *    of the last failure on the calling thread is prism_last_error(). No C++
 *    exception crosses this boundary.
 *  - `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *    legacy default stream). Work is enqueued on that stream; functions that
 *    return host data synchronise it. Asynchronous device errors surface at the
 *    next synchronising call (prism_sync, prism_get_*).
 *  - A voxel index v runs over the masked voxels of volume 0 in C order of
 *    (x, y, z), then volume 1, and so on ("mask order"). V = total voxels.
 *  - Raw per-voxel parameters, Q = 4K + 5 per voxel, in this order:
 *      [0]            s        S0 = softplus(s)
 *      [1 .. K+3]     logits   fractions = softmax over [csf, gm, wm_1..wm_K, res]
 *      [K+4 .. 4K+3]  v_k      3 components per fiber, d_k = v_k / max(|v_k|, 1e-12)
 *      [4K+4]         u        f_intra = sigmoid(u)
 *  - The handle owns every device buffer it allocates; caller buffers are only
 *    read during the call that receives them (init copies what it needs).
 *  - Handles are not thread-safe; distinct handles may be used concurrently.
 */
#ifndef PRISM_H
#define PRISM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum prism_status {
  PRISM_OK = 0,
  PRISM_E_INVALID_ARG = 1, /* NULL pointer, option out of range */
  PRISM_E_SHAPE = 2,       /* inconsistent sizes, empty mask, no b=0 measurement */
  PRISM_E_CUDA = 3,        /* a CUDA runtime call failed */
  PRISM_E_OOM = 4,         /* device allocation failed */
  PRISM_E_NONFINITE = 5,   /* non-finite input signal / b0, or the objective became NaN/Inf */
  PRISM_E_TIMEOUT = 6,     /* a bounded device-side wait gave up (status word set by a kernel) */
  PRISM_E_STATE = 7        /* call out of order (e.g. backward without forward), bad checkpoint */
} prism_status;

enum { PRISM_LOSS_MSE = 0, PRISM_LOSS_NLL = 1 };
enum { PRISM_MEM_HOST = 0, PRISM_MEM_DEVICE = 1 };
enum { PRISM_OPT_ADAM = 0, PRISM_OPT_RPROP = 1 };
enum { PRISM_MAX_K = 5, PRISM_BIAS_GRID = 8 };

/* One volume = one calibration / noise group (Sec. 2.3: b_lr, alpha_n, beta_n, sigma). */
typedef struct prism_volume {
  int32_t nx, ny, nz;     /* grid size, each >= 1 */
  int32_t n_meas;         /* N >= 1; at least one b <= 50 s/mm^2 (used for b0 normalisation) */
  int32_t mem;            /* PRISM_MEM_HOST or PRISM_MEM_DEVICE: where `signal` and `init` live */
  int32_t norm_count;     /* |M| that divides the MSE and the prior means (Eq. 8, Sec. 2.4): 0 = the
                             masked voxels of this mask. A caller that fits some whole patches of
                             a larger volume (a shard of it on one GPU) passes that volume's mask
                             restricted to those patches and the whole volume's masked count here;
                             without calibration and with the MSE, every voxel then follows the
                             whole-volume fit exactly (patches are independent problems).
                             E_SHAPE if 0 < norm_count < the masked voxels of this mask. */
  const uint8_t* mask;    /* HOST [nx][ny][nz], C order, nonzero = inside the brain mask */
  const float* signal;    /* [V_vol][N] raw magnitudes of the masked voxels in mask order */
  const float* bvals;     /* HOST [N] b-values, s/mm^2 (>= 0) */
  const float* bvecs;     /* HOST [N][3] gradient directions; rows with b > 50 must be unit (|g|-1| < 1e-3) */
  const float* init;      /* [V_vol][Q] raw initial parameters, or NULL for the seeded default */
} prism_volume;

typedef struct prism_options {
  int32_t K;              /* fibers per voxel, 1..5 */
  int32_t loss;           /* PRISM_LOSS_MSE (Eq. 8) or PRISM_LOSS_NLL (Eq. 9) */
  int32_t calibration;    /* 1: learn bias field + per-measurement affine (Sec. 2.3) */
  int32_t patch_dim;      /* spatial patch edge, 1..64; neighbour priors stay inside a patch */
  float lam_rep;          /* direction repulsion weight (Sec. 2.4), 0.01 */
  float lam_sparse;       /* L1 on minor fiber fractions, 0.02 */
  float tau;              /* minor-fraction threshold, 0.15 */
  float lam_sp;           /* Huber-Laplacian fraction smoothness (Eq. 7), 0 = off (paper default 0.01) */
  float huber_delta;      /* Huber transition, 0.05 */
  float lam_dir;          /* directional continuity, 0 = off (paper 0.005) */
  float lam_orphan;       /* orphan-WM suppression lam * mean exp(-S0/s_orphan) sum_k f_wm,k, 0 = off (paper 0.01) */
  float s_orphan;         /* S0 scale of orphan-WM suppression, 0.05 */
  float lam_order;        /* fiber ordering lam * mean sum_k max(0, f_wm,k+1 - f_wm,k), 0 = off (paper 0.01) */
  int32_t connectivity;   /* neighbourhood of the neighbour priors: 6 or 26 (Sec. 2.4) */
  float w_alpha, w_beta, w_blr, w_tv, tv_eps; /* calibration regularisers: 1e-3 each, eps 1e-6 */
  float sigma_init;       /* sigma start when a volume has < 2 b=0 measurements, 0.05 */
  float lr, beta1, beta2, eps; /* Adam: 1e-2, 0.9, 0.999, 1e-8; lr is also Rprop's initial step */
  int32_t optimizer;      /* PRISM_OPT_ADAM (default) or PRISM_OPT_RPROP, the paper's solver (Sec. 2.5) */
  float rprop_eta_minus;  /* Rprop step factor after a gradient sign change, 0.5 */
  float rprop_eta_plus;   /* Rprop step factor while the sign holds, 1.2 */
  float rprop_step_min, rprop_step_max; /* Rprop step bounds, 1e-6 and 50 */
  int32_t fused;          /* 1: persistent fused iteration kernel; 0: plain unfused per-patch launches */
  int32_t use_graph;      /* 1: replay the fused iteration from a CUDA graph */
  int32_t threads_per_voxel; /* 1, 4 or 16 (measurements split across lanes); 0 = automatic:
                                16 below 2,048 voxels, 4 below 32,768, else 1 except where
                                128-voxel tiles come to 0.75-1.25 waves of the fused kernel's
                                resident CTAs (then 4); prism_get_shape reports the choice */
  int32_t cta_threads;    /* plain path: 128 or 256 threads per CTA; 0 = automatic (the fused kernel uses 128) */
  int32_t autotune;       /* 1: time the candidate launch shapes at init and keep the fastest: lanes
                             per voxel 1 / 4 / 16 (or the forced value) and, with one lane, the shell
                             loop or the per-measurement loop; above about 311k voxels on a bounded
                             sample of each volume's fullest patches */
  int32_t seed;           /* seed of the default initialisation (init == NULL) */
  int32_t shells;         /* fused kernel, one thread per voxel, MSE, no calibration, K <= 3: 0 = take
                             the shell loop (per b-value shell work done once; needs every shell of
                             every volume to hold an even number of measurements), -1 = never */
  int32_t reserved[3];
} prism_options;

/* Fills `opt` with the paper's defaults (MSE, K = 3, no calibration, repulsion + sparsity). */
void prism_default_options(prism_options* opt);

typedef struct prism_handle prism_handle;

/*
 * Validates the volumes, b0-normalises the signal (Sec. 2.5), splits each mask
 * into patch_dim^3 patches and voxel tiles, packs the data for the kernels,
 * builds the per-measurement tables, and initialises parameters, Adam state and
 * (if requested) the CUDA graph. Allocates all device memory the fit needs.
 * Errors: E_INVALID_ARG, E_SHAPE (sizes, empty mask, no b=0), E_NONFINITE
 * (non-finite signal or non-positive b0 mean), E_OOM, E_CUDA.
 */
int prism_fit_init(const prism_volume* vols, int32_t n_vols, const prism_options* opt,
                   void* stream, prism_handle** out);

/* Enqueues n_iters >= 0 iterations (objective, gradient, Adam update). Asynchronous. */
int prism_step(prism_handle* h, int32_t n_iters, void* stream);

/* Synchronises `stream` and reports any device-side status (E_TIMEOUT, E_NONFINITE) or CUDA error. */
int prism_sync(prism_handle* h, void* stream);

/*
 * Check of the bounded device-side waits (the paper has no counterpart; for tests of the
 * error path). Enqueues one small kernel that waits, with the same bounded wait the fused
 * kernel uses for its bulk copies, on a barrier phase that nothing completes: no copy is
 * issued and nothing arrives, so nothing is left in flight. After max_polls polls
 * (1 .. 1,048,576) the wait gives up, the kernel sets the handle's timeout status and
 * returns; the next prism_sync returns PRISM_E_TIMEOUT, as every later one on this handle
 * does. The CUDA context and other handles stay usable. E_INVALID_ARG for a NULL handle or
 * max_polls out of range.
 */
int prism_wait_probe(prism_handle* h, int32_t max_polls, void* stream);

/* Sizes: total voxels V, groups, Q, total packed group-parameter floats, iterations done. */
int prism_info(const prism_handle* h, int64_t* n_vox, int32_t* n_groups, int32_t* q,
               int64_t* n_group_params, int64_t* iterations);

/*
 * Launch shape the handle runs with: lanes per voxel (1, 4 or 16; chosen at init from the
 * voxel count unless prism_options.threads_per_voxel forces one), voxels per tile, CTAs of
 * the persistent fused kernel (0 for a plain handle) and whether the fused kernel takes the
 * shell loop (1) or the per-measurement loop (0). Any output pointer may be NULL. The paper
 * has no counterpart: the shape is this implementation's. Errors: PRISM_E_INVALID_ARG for a
 * NULL handle.
 */
int prism_get_shape(const prism_handle* h, int32_t* threads_per_voxel, int32_t* tile_voxels, int32_t* fused_grid,
                    int32_t* shell_loop);

/* Raw parameters [V][Q] in mask order, to/from host or device memory (per `mem`). */
int prism_get_params(prism_handle* h, float* out, int32_t mem, void* stream);
int prism_set_params(prism_handle* h, const float* in, int32_t mem, void* stream);

/*
 * Readout of the fitted fibers (Sec. 3 "Configuration": fiber directions are used directly
 * as peaks): unit directions dirs [V][K][3], fractions fracs [V][K+3] ([csf, gm, wm_1..wm_K,
 * res]) and peak flags peaks [V][K] (1 when the fiber's share of the white-matter fraction
 * is >= rel_thresh, e.g. 0.15), mask order, in `mem` memory. Any output may be NULL.
 * E_INVALID_ARG for rel_thresh outside [0, 1].
 */
int prism_get_fibers(prism_handle* h, float* dirs, float* fracs, uint8_t* peaks, float rel_thresh,
                     int32_t mem, void* stream);

/*
 * Whole-volume fit in overlapping slabs (Sec. 3 "Configuration": the whole brain is fitted
 * as 30-slice slabs with a 5-slice overlap, stitched by weighted averaging). `vol` is split
 * along its last axis into slabs of `slab` slices advancing by slab - overlap, the last one
 * reaching the last slice; every non-empty slab becomes one volume of a handle initialised as
 * by prism_fit_init (its own sigma and calibration; neighbour priors stay inside the slab).
 * The slab signals (and `init` rows) are gathered on the device from vol->signal in `vol->mem`
 * memory; the caller's buffers are not kept. Step the handle as usual, then read the
 * whole-volume maps with prism_stitch_slabs. E_INVALID_ARG for slab < 1, overlap < 0 or
 * 2 * overlap > slab, E_SHAPE for an empty mask, plus every error of prism_fit_init.
 */
int prism_fit_init_slabs(const prism_volume* vol, int32_t slab, int32_t overlap, const prism_options* opt,
                         void* stream, prism_handle** out);

/*
 * Whole-volume maps of a handle made by prism_fit_init_slabs, in the original volume's mask
 * order and `mem` memory: S0 [V], fractions [V][K+3] ([csf, gm, wm_1..wm_K, res]), f_intra [V],
 * unit directions [V][K][3]; any output may be NULL. A voxel in one slab takes that slab's
 * estimate. In an overlap the later slab's weight ramps linearly across the overlapping
 * slices, w = (z - z0 + 1/2) / overlap; its fibers are matched to the earlier slab's by the
 * permutation maximising sum_k |d_k . d'_pi(k)| (FP64, first maximum in lexicographic order),
 * flipped into the same hemisphere, and S0, fractions, f_intra and directions are averaged
 * (directions renormalised). E_STATE for a handle not made by prism_fit_init_slabs.
 */
int prism_stitch_slabs(prism_handle* h, float* s0, float* fracs, float* fin, float* dirs, int32_t mem,
                       void* stream);

/*
 * Packed group parameters. Group g occupies [off[4g], off[4g+4]) of the packed
 * float array: sigma_log at off[4g], alpha[N_g] at off[4g+1], beta[N_g] at
 * off[4g+2], b_lr[8][8][8] (C order) at off[4g+3]; off[4G] = total. `off` is a
 * HOST int64 array of 4G+1 entries.
 */
int prism_group_layout(const prism_handle* h, int64_t* off);
int prism_get_groups(prism_handle* h, float* out, int32_t mem, void* stream);
int prism_set_groups(prism_handle* h, const float* in, int32_t mem, void* stream);

/*
 * Objective per group J_g (data term + priors + calibration regularisers,
 * Sec. 2.5) evaluated at the parameters before the most recent update, as
 * double. `hist` (HOST, may be NULL) receives up to `max_iters` x G values of
 * the most recent iterations, oldest first; `*n_written` the iteration count.
 */
int prism_get_loss(prism_handle* h, double* loss, double* hist, int32_t max_iters,
                   int32_t* n_written);

/*
 * Forward evaluation at `theta` (DEVICE [V][Q], or NULL = current parameters)
 * and `groups` (DEVICE packed, or NULL = current): synthesis, calibration and
 * data term, plus the prior values. A given theta / groups becomes the handle's
 * current parameters (as by prism_set_params / prism_set_groups). Writes y_hat (DEVICE, NULL to skip; group g
 * at offset sum_{g'<g} V_g' N_g', rows [V_g][N_g] in mask order) and J_g
 * (DEVICE double [G]). Keeps the residual derivative dL/dy_hat (V x N, not the
 * V x N x K compartment terms) for prism_backward.
 */
int prism_forward(prism_handle* h, const float* theta, const float* groups, float* yhat,
                  double* loss, void* stream);

/*
 * Gradient of the objective at the point of the last prism_forward: recomputes
 * the compartment exponentials, then the adjoint of synthesis, calibration,
 * data term and priors. grad_theta DEVICE [V][Q]; grad_groups DEVICE packed
 * (NULL to skip). E_STATE without a preceding forward.
 */
int prism_backward(prism_handle* h, float* grad_theta, float* grad_groups, void* stream);

/*
 * Timing probe: enqueues n_iters >= 1 fused iterations WITHOUT the CUDA graph, with CUDA
 * events on `stream` around each kernel class, waits for them, and writes the average
 * milliseconds per iteration to ms_out (HOST float[4]): [0] the fused iteration kernel,
 * [1] the neighbour-prior preparation kernel, [2] the group kernels (bias gradient,
 * reductions, group Adam; launched only with calibration -- otherwise the fused kernel's
 * last CTA finalises the groups and [2] is 0), [3] the whole iteration. The iterations are
 * real updates.
 * E_STATE on a handle created with fused = 0.
 */
int prism_profile(prism_handle* h, int32_t n_iters, void* stream, float* ms_out);

/*
 * Pipe microbenchmark for roofline denominators: kind 0 = FP32 fused multiply-add,
 * 1 = packed float2 FMA, 2 = special-function 2^x (ex2.approx), 3 = FP64 FMA. Runs a
 * fixed amount of independent dependency chains on every SM of the current device and
 * writes the achieved rate to *ops_per_s (flops, FMA = 2; for kind 2 exponentials/s).
 * Synchronous; allocates a small sink buffer.
 */
int prism_microbench(int32_t kind, double* ops_per_s, void* stream);

/* Checkpoint: parameters, Adam moments, step counter and group state as one blob. */
int prism_state_size(const prism_handle* h, int64_t* bytes);
int prism_get_state(prism_handle* h, void* host_buf, int64_t bytes, void* stream);
int prism_set_state(prism_handle* h, const void* host_buf, int64_t bytes, void* stream);

/*
 * One-call fit: init + n_iters iterations + readout + destroy. params_out
 * [V][Q] and loss_out [G] (double) live in `out_mem` memory (either may be
 * NULL). Synchronous.
 */
int prism_fit(const prism_volume* vols, int32_t n_vols, const prism_options* opt,
              int32_t n_iters, float* params_out, double* loss_out, int32_t out_mem,
              void* stream);

/*
 * Allocation-free objective and gradient (the paper has no counterpart of this call).
 *
 * For callers that must not allocate device memory where they evaluate the fit: code
 * running inside a framework that owns the whole device memory pool, real-time
 * pipelines that reserve all memory up front because cudaMalloc / cudaFree can
 * synchronise the device, and plugins whose host forbids allocations outside its own
 * allocator. It needs no handle and calls no cudaMalloc, cudaFree or allocating library
 * routine: beyond the caller's buffers it uses one fixed 128 KiB array inside the
 * library, which every GPU that loads the library keeps until the process exits.
 *
 * Evaluates, for n_vox voxels forming one group, J = (sum of squared differences between
 * predicted and measured signal over all voxels and measurements) / n_vox + lam_rep * mean
 * fiber-direction repulsion + lam_sparse * mean minor-fraction sparsity, without
 * calibration or neighbour priors, on raw signal rows that it divides by each voxel's mean
 * b <= 50 signal itself, and its gradient -- the same values prism_forward and
 * prism_backward give for that problem.
 *   signal  DEVICE [n_vox][n_meas] raw magnitudes;  theta DEVICE [n_vox][4K+5] raw parameters
 *   bvals   HOST [n_meas];  bvecs HOST [n_meas][3]
 *   grad    DEVICE [n_vox][4K+5] (written);  loss DEVICE double[1] (written)
 * Limits: 1 <= n_vox <= 1,048,576, 1 <= n_meas <= 1024, 1 <= K <= 5 (E_SHAPE /
 * E_INVALID_ARG otherwise, before any device work); at least one b <= 50 measurement;
 * b-values finite and >= 0, b-vectors finite and of unit length where b > 50, as for
 * prism_fit_init (E_INVALID_ARG). The signal is read on the GPU after the call returns, so
 * a voxel whose mean b <= 50 signal is not positive and finite (which prism_fit_init
 * refuses with E_NONFINITE) is reported in the outputs instead: its gradient row and the
 * loss are NaN; the other rows are computed as usual.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress).
 * Every call shares the array and leaves its contents behind (it clears what must start
 * at zero itself), so two calls whose GPU work overlaps on the same device (for example
 * on two streams) race with each other: serialise them.
 */
int prism_grad_noalloc(const float* signal, const float* bvals, const float* bvecs, const float* theta,
                       int64_t n_vox, int32_t n_meas, int32_t K, float lam_rep, float lam_sparse,
                       float tau, float* grad, double* loss, void* stream);

/* Frees every device buffer and graph of the handle. NULL is a no-op. */
void prism_fit_destroy(prism_handle* h);

/* Message of the last failure on this thread ("" if none). Valid until the next call. */
const char* prism_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PRISM_H */
