// C-ABI implementation of the PRISM fitting library (host side).
//
// Responsibilities: argument validation, the spatial work decomposition (volumes ->
// patch_dim^3 patches -> voxel tiles), packing of the b0-normalised signal (Sec. 2.5),
// device workspace, the fused (persistent kernel, CUDA graph) and plain (per-patch
// launches) iteration drivers, the forward / backward evaluation behind the autograd
// binding, checkpointing and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <thread>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "host_pool.h"
#include "prism.h"
#include "prism_kernels.cuh"
#include "prism_launch.h"

using namespace prism;

namespace prism {
const KernelSet& kernels_k1();
const KernelSet& kernels_k2();
const KernelSet& kernels_k3();
const KernelSet& kernels_k4();
const KernelSet& kernels_k5();
const KernelSet& kernels_for_k(int K) {
  switch (K) {
    case 1: return kernels_k1();
    case 2: return kernels_k2();
    case 3: return kernels_k3();
    case 4: return kernels_k4();
    default: return kernels_k5();
  }
}
}  // namespace prism

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? PRISM_E_OOM : PRISM_E_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

constexpr int kSplitTiles = 64;
constexpr int kHistLen = 4096;
constexpr int kGraphUnroll = 16;
constexpr uint32_t kStateMagic = 0x50524953u;   // "PRIS"

struct PatchRange {
  int tb, te;
};

}  // namespace

struct prism_handle {
  prism_options opt{};
  int K = 0, Q = 0, XF = 0, TPV = 1, NT = 128, TV = 128;
  int G = 0, Vpad = 0, ntiles = 0, Nmax = 0, max_e = 0, max_split = 0;
  int64_t V = 0, GP = 0, iters = 0, ypack_len = 0, tab_rows = 0, ab_len = 0, yhat_len = 0;
  bool cal = false, nb = false;
  std::vector<GroupDev> groups;
  std::vector<Tile> tiles;
  std::vector<PatchRange> patches;
  std::vector<int64_t> vox0, gp_layout, yhat_off;
  std::vector<void*> allocs;
  // device buffers
  Tile* d_tiles = nullptr;
  int32_t* d_tile_order = nullptr;   // the fused kernel's queue order (see tile_queue_order)
  GroupDev* d_groups = nullptr;
  float *d_y = nullptr, *d_theta = nullptr, *d_m = nullptr, *d_v = nullptr, *d_xf = nullptr;
  float *d_hsp = nullptr, *d_lp = nullptr, *d_pg = nullptr, *d_gU = nullptr, *d_tile_ab = nullptr;
  float *d_gparams = nullptr, *d_gm = nullptr, *d_gv = nullptr;
  float *d_yhat = nullptr, *d_r = nullptr, *d_grad = nullptr;
  int32_t *d_nbr = nullptr, *d_queue = nullptr, *d_done = nullptr, *d_step = nullptr, *d_status = nullptr;
  float* d_adamc = nullptr;
  int32_t *d_slot_of_vox = nullptr, *d_vox_of_slot = nullptr, *d_slot_of_grid = nullptr;
  int32_t *d_split_off = nullptr, *d_counters = nullptr;
  uint32_t *d_vcoord = nullptr, *d_vflag = nullptr;
  int64_t* d_row_off = nullptr;
  int32_t* d_order = nullptr;          // [tab_rows] table position -> caller's measurement index
  // slab fits (prism_fit_init_slabs): per voxel of the whole volume, its source voxel(s) in
  // the handle and the weight of the second source
  bool slabbed = false;
  std::vector<int64_t> st_src0, st_src1;
  std::vector<float> st_w1;
  std::vector<int32_t> order;          // host copy
  MeasRow* d_table = nullptr;
  MeasPair* d_table2 = nullptr;
  int64_t tab2_pairs = 0;
  // shell loop: per-group gradient rows and shells (host copies built by the plan)
  std::vector<float> gtab;
  std::vector<ShellRun> runs;
  bool shells_even = true;             // every group's shells hold an even number of measurements
  bool shell = false;                  // the fused kernel takes the shell loop
  float* d_gtab = nullptr;
  ShellRun* d_runs = nullptr;
  double *d_tile_red = nullptr, *d_part2 = nullptr, *d_gred = nullptr, *d_gloss = nullptr;
  double* d_bscratch = nullptr;      // bias-gradient partial contractions (calibration only)
  int64_t* d_bs_off = nullptr;       // [G][2] offsets into d_bscratch
  int max_nx = 0, max_ny = 0;
  int32_t* d_gdone = nullptr;
  double *d_gprior = nullptr, *d_hist = nullptr;
  IterArgs ia{};
  GroupArgs ga{};
  const KernelSet* ks = nullptr;
  int fused_grid = 0;
  size_t fused_smem = 0, adj_smem = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t g1 = nullptr, gU = nullptr;
  bool forward_done = false;

  template <typename T>
  int alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_fail(e, "cudaMalloc");
    }
    allocs.push_back(q);
    *p = static_cast<T*>(q);
    return PRISM_OK;
  }
  ~prism_handle() {
    if (g1) cudaGraphExecDestroy(g1);
    if (gU) cudaGraphExecDestroy(gU);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (void* p : allocs) cudaFree(p);
  }
};

extern "C" void prism_default_options(prism_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->K = 3;
  o->loss = PRISM_LOSS_MSE;
  o->calibration = 0;
  o->patch_dim = 16;
  o->lam_rep = 0.01f;
  o->lam_sparse = 0.02f;
  o->tau = 0.15f;
  o->lam_sp = 0.f;
  o->huber_delta = 0.05f;
  o->lam_dir = 0.f;
  o->lam_orphan = 0.f;
  o->s_orphan = 0.05f;
  o->lam_order = 0.f;
  o->connectivity = 6;
  o->w_alpha = o->w_beta = o->w_blr = o->w_tv = 1e-3f;
  o->tv_eps = 1e-6f;
  o->sigma_init = 0.05f;
  o->lr = 1e-2f;
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-8f;
  o->optimizer = PRISM_OPT_ADAM;
  o->rprop_eta_minus = 0.5f;
  o->rprop_eta_plus = 1.2f;
  o->rprop_step_min = 1e-6f;
  o->rprop_step_max = 50.f;
  o->fused = 1;
  o->use_graph = 1;
  o->threads_per_voxel = 0;
  o->cta_threads = 0;
  o->autotune = 0;
  o->seed = 0;
}

extern "C" const char* prism_last_error(void) { return g_err.c_str(); }

// Lets other translation units of the library report through prism_last_error().
int prism_record_error(int code, const char* msg) { return fail(code, msg); }

namespace {

bool finite_nonneg(float x) { return std::isfinite(x) && x >= 0.f; }

int validate_options(const prism_options& o) {
  if (o.K < 1 || o.K > PRISM_MAX_K) return fail(PRISM_E_INVALID_ARG, "K must be in 1..5");
  if (o.loss != PRISM_LOSS_MSE && o.loss != PRISM_LOSS_NLL) return fail(PRISM_E_INVALID_ARG, "loss must be MSE (0) or NLL (1)");
  if (o.calibration != 0 && o.calibration != 1) return fail(PRISM_E_INVALID_ARG, "calibration must be 0 or 1");
  if (o.patch_dim < 1 || o.patch_dim > 64) return fail(PRISM_E_INVALID_ARG, "patch_dim must be in 1..64");
  const float nn[] = {o.lam_rep, o.lam_sparse, o.tau, o.lam_sp, o.lam_dir, o.w_alpha, o.w_beta, o.w_blr, o.w_tv,
                      o.lam_orphan, o.lam_order};
  for (float x : nn)
    if (!finite_nonneg(x)) return fail(PRISM_E_INVALID_ARG, "prior weights and tau must be finite and >= 0");
  if (!(o.huber_delta > 0.f) || !std::isfinite(o.huber_delta)) return fail(PRISM_E_INVALID_ARG, "huber_delta must be > 0");
  if (!(o.tv_eps > 0.f)) return fail(PRISM_E_INVALID_ARG, "tv_eps must be > 0");
  if (!(o.s_orphan > 0.f) || !std::isfinite(o.s_orphan)) return fail(PRISM_E_INVALID_ARG, "s_orphan must be > 0");
  if (o.connectivity != 6 && o.connectivity != 26) return fail(PRISM_E_INVALID_ARG, "connectivity must be 6 or 26");
  if (!(o.sigma_init > 0.f) || !std::isfinite(o.sigma_init)) return fail(PRISM_E_INVALID_ARG, "sigma_init must be > 0");
  if (!(o.lr > 0.f) || !std::isfinite(o.lr)) return fail(PRISM_E_INVALID_ARG, "lr must be > 0");
  if (!(o.beta1 >= 0.f && o.beta1 < 1.f) || !(o.beta2 >= 0.f && o.beta2 < 1.f))
    return fail(PRISM_E_INVALID_ARG, "Adam betas must be in [0, 1)");
  if (!(o.eps > 0.f)) return fail(PRISM_E_INVALID_ARG, "Adam eps must be > 0");
  if (o.optimizer != PRISM_OPT_ADAM && o.optimizer != PRISM_OPT_RPROP)
    return fail(PRISM_E_INVALID_ARG, "optimizer must be PRISM_OPT_ADAM or PRISM_OPT_RPROP");
  if (o.optimizer == PRISM_OPT_RPROP &&
      !(o.rprop_eta_minus > 0.f && o.rprop_eta_minus < 1.f && o.rprop_eta_plus > 1.f && o.rprop_step_min > 0.f &&
        o.rprop_step_max >= o.rprop_step_min && o.lr >= o.rprop_step_min && o.lr <= o.rprop_step_max))
    return fail(PRISM_E_INVALID_ARG, "Rprop needs 0 < eta_minus < 1 < eta_plus and 0 < step_min <= lr <= step_max");
  if (o.threads_per_voxel != 0 && o.threads_per_voxel != 1 && o.threads_per_voxel != 4 && o.threads_per_voxel != 16)
    return fail(PRISM_E_INVALID_ARG, "threads_per_voxel must be 0, 1, 4 or 16");
  if (o.shells != 0 && o.shells != -1) return fail(PRISM_E_INVALID_ARG, "shells must be 0 (automatic) or -1 (off)");
  if (o.cta_threads != 0 && o.cta_threads != 128 && o.cta_threads != 256)
    return fail(PRISM_E_INVALID_ARG, "cta_threads must be 0, 128 or 256");
  return PRISM_OK;
}

int validate_volume(const prism_volume& v, int g) {
  const std::string w = "volume " + std::to_string(g) + ": ";
  if (!v.mask || !v.signal || !v.bvals || !v.bvecs) return fail(PRISM_E_INVALID_ARG, w + "mask, signal, bvals and bvecs are required");
  if (v.nx < 1 || v.ny < 1 || v.nz < 1 || v.nx > 1023 || v.ny > 1023 || v.nz > 1023)
    return fail(PRISM_E_SHAPE, w + "grid sizes must be in 1..1023");
  if (v.n_meas < 1 || v.n_meas > 1024) return fail(PRISM_E_SHAPE, w + "n_meas must be in 1..1024");
  if (v.mem != PRISM_MEM_HOST && v.mem != PRISM_MEM_DEVICE) return fail(PRISM_E_INVALID_ARG, w + "mem must be HOST or DEVICE");
  int nb0 = 0;
  for (int n = 0; n < v.n_meas; ++n) {
    const float b = v.bvals[n];
    if (!std::isfinite(b) || b < 0.f) return fail(PRISM_E_INVALID_ARG, w + "b-values must be finite and >= 0");
    const float gx = v.bvecs[3 * n], gy = v.bvecs[3 * n + 1], gz = v.bvecs[3 * n + 2];
    if (!std::isfinite(gx) || !std::isfinite(gy) || !std::isfinite(gz)) return fail(PRISM_E_INVALID_ARG, w + "non-finite b-vector");
    if (b <= 50.f) {
      ++nb0;
    } else if (std::fabs(std::sqrt(gx * gx + gy * gy + gz * gz) - 1.f) > 1e-3f) {
      return fail(PRISM_E_INVALID_ARG, w + "b-vector " + std::to_string(n) + " of a b > 50 measurement is not unit length");
    }
  }
  if (nb0 == 0) return fail(PRISM_E_SHAPE, w + "no b <= 50 measurement to normalise by");
  return PRISM_OK;
}

void fill_args(prism_handle* h) {
  IterArgs& a = h->ia;
  a.Q = h->Q;
  a.Vpad = h->Vpad;
  a.TV = h->TV;
  a.VW = 32 / h->TPV;
  a.ntiles = h->ntiles;
  a.Nmax = h->Nmax;
  a.G = h->G;
  a.tiles = h->d_tiles;
  a.tile_order = h->d_tile_order;
  a.groups = h->d_groups;
  a.y = h->d_y;
  a.theta = h->d_theta;
  a.m = h->d_m;
  a.v = h->d_v;
  a.xf = h->d_xf;
  a.hsp = h->d_hsp;
  a.lp = h->d_lp;
  a.pg = h->d_pg;
  a.nbr = h->d_nbr;
  a.vcoord = h->d_vcoord;
  a.vflag = h->d_vflag;
  a.table = h->d_table;
  a.table2 = h->d_table2;
  a.gtab = h->d_gtab;
  a.runs = h->d_runs;
  a.gparams = h->d_gparams;
  a.gU = h->d_gU;
  a.tile_ab = h->d_tile_ab;
  a.tile_red = h->d_tile_red;
  a.queue = h->d_queue;
  a.done = h->d_done;
  a.step = h->d_step;
  a.adamc = h->d_adamc;
  a.status = h->d_status;
  const prism_options& o = h->opt;
  a.lam_rep = o.lam_rep;
  a.lam_sparse = o.lam_sparse;
  a.tau = o.tau;
  a.lam_sp = o.lam_sp;
  a.huber_delta = o.huber_delta;
  a.lam_dir = o.lam_dir;
  a.w_tv = o.calibration ? o.w_tv : 0.f;
  a.tv_eps = o.tv_eps;
  a.lr = o.lr;
  a.beta1 = o.beta1;
  a.beta2 = o.beta2;
  a.eps = o.eps;
  a.optimizer = o.optimizer;
  a.eta_minus = o.rprop_eta_minus;
  a.eta_plus = o.rprop_eta_plus;
  a.step_min = o.rprop_step_min;
  a.step_max = o.rprop_step_max;
  a.nb_priors = h->nb ? 1 : 0;
  a.pdl = 1;
  a.n_nbr = o.connectivity;
  a.lam_orphan = o.lam_orphan;
  a.inv_s_orphan = 1.f / o.s_orphan;
  a.lam_order = o.lam_order;
  a.fold_groups = h->cal ? 0 : 1;
  a.loss_mode = o.loss;
  a.hist_len = kHistLen;
  a.gparams_rw = h->d_gparams;
  a.gm = h->d_gm;
  a.gv = h->d_gv;
  a.gloss = h->d_gloss;
  a.hist = h->d_hist;

  GroupArgs& g = h->ga;
  g.G = h->G;
  g.max_split = h->max_split;
  g.split_tiles = kSplitTiles;
  g.max_e = h->max_e;
  g.split_off = h->d_split_off;
  g.part2 = h->d_part2;
  g.counters = h->d_counters;
  g.gred = h->d_gred;
  g.gloss = h->d_gloss;
  g.gprior = h->d_gprior;
  g.gm = h->d_gm;
  g.gv = h->d_gv;
  g.gparams = h->d_gparams;
  g.table = h->d_table;
  g.table2 = h->d_table2;
  g.bscratch = h->d_bscratch;
  g.gdone = h->d_gdone;
  g.bs_off = h->d_bs_off;
  g.max_nx = h->max_nx;
  g.max_ny = h->max_ny;
  g.slot_of_grid = h->d_slot_of_grid;
  g.hist = h->d_hist;
  g.hist_len = kHistLen;
  g.gexport = nullptr;
  g.loss_mode = o.loss;
  g.w_alpha = o.w_alpha;
  g.w_beta = o.w_beta;
  g.w_blr = o.w_blr;
}

// Enqueues one fused iteration.
int enqueue_fused_iter(prism_handle* h, cudaStream_t st) {
  const IterArgs& a = h->ia;
  if (h->opt.lam_sp > 0.f) CK(h->ks->prior_prep(a, 0, h->ntiles, st));
  if (h->nb) CK(h->ks->prior_grad(a, 0, h->ntiles, st));
  CK(h->ks->fused(a, h->opt.loss, h->cal ? 1 : 0, h->TPV, h->shell ? 1 : 0, h->fused_grid, h->NT, h->fused_smem, st));
  if (h->cal) {   // without calibration the fused kernel's last CTA finalises the groups
    CK(launch_bias_grad(a, h->ga, st));
    CK(launch_group_reduce(a, h->ga, 1 | 2, st));
    CK(launch_group_adam(a, h->ga, 1 | 2, st));
  }
  return PRISM_OK;
}

// Enqueues one plain iteration: separate synthesis, loss, adjoint, prior and Adam launches
// per patch, then the group update.
int enqueue_plain_iter(prism_handle* h, cudaStream_t st) {
  const IterArgs& a = h->ia;
  const int cal = h->cal ? 1 : 0;
  for (const PatchRange& pr : h->patches) {
    PlainArgs p{h->d_yhat, h->d_r, h->d_grad, pr.tb, pr.te, 3};
    CK(h->ks->transform(a, pr.tb, pr.te, st));
    CK(h->ks->synth(a, p, cal, h->TPV, h->NT, st));
    CK(launch_loss(a, p, h->opt.loss, st));
    if (h->opt.lam_sp > 0.f) CK(h->ks->prior_prep(a, pr.tb, pr.te, st));
    CK(h->ks->adjoint(a, p, cal, h->TPV, h->NT, h->adj_smem, st));
    CK(h->ks->prior(a, p, st));
    CK(launch_adam_voxel(a, p, st));
  }
  if (h->cal) CK(launch_bias_grad(a, h->ga, st));
  CK(launch_group_reduce(a, h->ga, 1 | (h->cal ? 2 : 0), st));
  CK(launch_group_adam(a, h->ga, 1 | 2, st));
  return PRISM_OK;
}

int capture_graph(prism_handle* h, int iters, cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = PRISM_OK;
  for (int i = 0; i < iters && rc == PRISM_OK; ++i) rc = enqueue_fused_iter(h, h->cap_stream);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
  if (rc != PRISM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return PRISM_OK;
}

// Host-side plan of volumes -> patches -> tiles, neighbours and flags.
// Internal measurement order of one group, appended to `order` (table position -> the
// caller's index). Without calibration the measurements are sorted by b-value (stable): the
// b = 0 ones come first, so that the packed path can take their pairs without the fiber terms
// (every E of Eqs. 4-5 is 1 at b = 0), and equal b-values form runs (shells) for the shell
// loop. With calibration, whose alpha_n / beta_n are indexed by measurement, the order is the
// caller's. Returns the number of leading pairs whose two measurements have b = 0.
static int32_t meas_order(const prism_volume& v, bool cal, std::vector<int32_t>& order) {
  const int N = v.n_meas;
  if (cal) {
    for (int n = 0; n < N; ++n) order.push_back(n);
    return 0;
  }
  std::vector<int32_t> idx(N);
  for (int n = 0; n < N; ++n) idx[n] = n;
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return v.bvals[a] < v.bvals[b]; });
  int nz = 0;
  for (int n = 0; n < N; ++n) nz += v.bvals[n] == 0.f;
  order.insert(order.end(), idx.begin(), idx.end());
  return nz / 2;
}

// The fiber model's fixed diffusivities (Eq. 5, mm^2/s) and log2(e), for the shell loop's
// host-side constants.
constexpr double kDpar = 1.7e-3, kDperp = 0.4e-3, kLog2e = 1.4426950408889634;

// Shells of one group in table order (runs of equal b-value) with the constants of the
// shell loop (ShellRun); false when a shell holds an odd number of measurements (a pair would
// straddle two shells) or there are more than kMaxRuns shells.
static bool shell_runs(const prism_volume& v, const int32_t* ord, std::vector<ShellRun>& runs) {
  const int N = v.n_meas;
  bool ok = true;
  int n0 = 0, nr = 0;
  while (n0 < N) {
    const float b = v.bvals[ord[n0]];
    int n1 = n0 + 1;
    while (n1 < N && v.bvals[ord[n1]] == b) ++n1;
    if ((n1 - n0) % 2 != 0) ok = false;
    ShellRun r{};
    r.p0 = n0 / 2;
    r.p1 = n1 / 2;
    r.b0 = (b == 0.f) ? 1 : 0;
    const double bd = b;
    r.ecsf = static_cast<float>(std::exp(-bd * 3.0e-3));   // Eq. 4
    r.egm = static_cast<float>(std::exp(-bd * 0.9e-3));
    r.eres = static_cast<float>(std::exp(-bd * 0.2e-3));
    r.nbperp = static_cast<float>(-bd * kDperp * kLog2e);
    runs.push_back(r);
    ++nr;
    n0 = n1;
  }
  return ok && nr <= kMaxRuns;
}

// Runs fn(begin, end) over [0, n) split into contiguous chunks on the process's host worker
// pool (up to 16 threads with the caller; one chunk, on the calling thread, below
// `min_per_thread` items per thread, or when the pool is busy or absent).
template <typename F>
static void parallel_chunks(int64_t n, int64_t min_per_thread, F fn) {
  HostPool* pool = HostPool::get();
  int64_t nt = pool ? pool->threads() : 1;
  nt = std::max<int64_t>(1, std::min<int64_t>(nt, n / std::max<int64_t>(min_per_thread, 1)));
  if (nt > 1 && pool->run(n, static_cast<int>(nt), HostPool::Fn(fn))) return;
  fn(int64_t{0}, n);
}

// Order in which the fused kernel's queue hands out tiles: every full tile in plan order
// (volumes stay contiguous, so the measurement table rarely changes), then the partial tiles
// by decreasing voxel count. The last tiles of an iteration are then the cheapest, which
// shortens the tail where some CTAs are idle.
static std::vector<int32_t> tile_queue_order(const std::vector<Tile>& tiles, int TV) {
  std::vector<int32_t> order, part;
  order.reserve(tiles.size());
  for (size_t t = 0; t < tiles.size(); ++t) {
    if (tiles[t].count == TV) order.push_back(static_cast<int32_t>(t));
    else part.push_back(static_cast<int32_t>(t));
  }
  std::stable_sort(part.begin(), part.end(), [&](int32_t a, int32_t b) { return tiles[a].count > tiles[b].count; });
  order.insert(order.end(), part.begin(), part.end());
  return order;
}

// A vector whose elements start uninitialised: the plan's large index tables are written in
// full by its parallel passes, so a serial fill first would only add a pass over them.
template <typename T>
struct NoFillAlloc : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoFillAlloc<U>;
  };
  NoFillAlloc() = default;
  template <typename U>
  NoFillAlloc(const NoFillAlloc<U>&) noexcept {}
  template <typename U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <typename U, typename... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
template <typename T>
using RawVec = std::vector<T, NoFillAlloc<T>>;

struct Plan {
  RawVec<int32_t> slot_of_vox, slot_of_grid;
  RawVec<int64_t> row_off;
};

int build_plan(prism_handle* h, const prism_volume* vols, int n_vols, Plan& pl) {
  const int P = h->opt.patch_dim;
  const int TV = h->TV;
  h->G = n_vols;
  h->groups.assign(n_vols, GroupDev{});
  h->vox0.assign(n_vols + 1, 0);
  h->gp_layout.assign(4 * static_cast<size_t>(n_vols) + 1, 0);
  h->yhat_off.assign(n_vols + 1, 0);
  // counts
  int64_t Vtot = 0, grid_tot = 0;
  std::vector<RawVec<int32_t>> vidx(n_vols);
  for (int g = 0; g < n_vols; ++g) {
    const prism_volume& v = vols[g];
    const int64_t ng = static_cast<int64_t>(v.nx) * v.ny * v.nz;
    vidx[g].resize(ng);
    // mask-order index of every grid position (-1 outside the mask): chunk counts, then chunk
    // offsets
    constexpr int64_t kChunkN = 1 << 18;
    const int64_t nch = (ng + kChunkN - 1) / kChunkN;
    std::vector<int32_t> cc(nch + 1, 0);
    parallel_chunks(nch, 1, [&](int64_t b, int64_t e) {
      for (int64_t k = b; k < e; ++k) {
        int32_t n = 0;
        for (int64_t i = k * kChunkN; i < std::min(ng, (k + 1) * kChunkN); ++i) n += v.mask[i] != 0;
        cc[k + 1] = n;
      }
    });
    for (int64_t k = 0; k < nch; ++k) cc[k + 1] += cc[k];
    parallel_chunks(nch, 1, [&](int64_t b, int64_t e) {
      for (int64_t k = b; k < e; ++k) {
        int32_t n = cc[k];
        for (int64_t i = k * kChunkN; i < std::min(ng, (k + 1) * kChunkN); ++i) vidx[g][i] = v.mask[i] ? n++ : -1;
      }
    });
    const int32_t c = cc[nch];
    if (c == 0) return fail(PRISM_E_SHAPE, "volume " + std::to_string(g) + ": empty mask");
    if (v.norm_count != 0 && v.norm_count < c)
      return fail(PRISM_E_SHAPE, "volume " + std::to_string(g) + ": norm_count " + std::to_string(v.norm_count) +
                                     " is below the " + std::to_string(c) + " masked voxels");
    h->vox0[g] = Vtot;
    Vtot += c;
    h->groups[g].grid_off = grid_tot;
    grid_tot += ng;
  }
  h->vox0[n_vols] = Vtot;
  h->V = Vtot;
  // every entry of the three tables is written by pass 2 below
  pl.slot_of_vox.resize(Vtot);
  pl.row_off.resize(Vtot);
  pl.slot_of_grid.resize(grid_tot);
  // tiles
  int64_t yoff = 0, aboff = 0, tab = 0, gp = 0, yh = 0;
  int Nmax = 0;
  for (int g = 0; g < n_vols; ++g) {
    const prism_volume& v = vols[g];
    GroupDev& gr = h->groups[g];
    gr.nx = v.nx;
    gr.ny = v.ny;
    gr.nz = v.nz;
    gr.N = v.n_meas;
    gr.N4 = (v.n_meas + 3) / 4 * 4;
    gr.n_vox = static_cast<int32_t>(h->vox0[g + 1] - h->vox0[g]);
    gr.inv_M = 1.f / static_cast<float>(v.norm_count > 0 ? v.norm_count : gr.n_vox);
    gr.calib = h->cal ? 1 : 0;
    gr.table_off = static_cast<int32_t>(tab);
    gr.nb0p = meas_order(v, h->cal, h->order);
    {
      // shells and gradient rows of the group's table order (shell loop)
      const int32_t* ord = h->order.data() + tab;
      gr.run_off = static_cast<int32_t>(h->runs.size());
      if (!shell_runs(v, ord, h->runs)) h->shells_even = false;
      gr.n_runs = static_cast<int32_t>(h->runs.size()) - gr.run_off;
      const int NPg = (v.n_meas + 3) & ~3;
      gr.gtab_off = static_cast<int32_t>(h->gtab.size());
      h->gtab.resize(h->gtab.size() + 3 * static_cast<size_t>(NPg), 0.f);
      float* gt = h->gtab.data() + gr.gtab_off;
      // the scaled directions g' = s g, s = sqrt(b D_par log2 e) (Eq. 5: c' = s c = g' . d), per
      // pair p: {g'_x(2p), g'_x(2p+1), g'_y(2p), g'_y(2p+1)} at 4p, then g'_z of every measurement
      // from 2 NP on (one 16-byte and one 8-byte shared-memory load per pair)
      for (int n = 0; n < v.n_meas; ++n) {
        const int p = n / 2, h = n % 2;
        const double s = std::sqrt(static_cast<double>(v.bvals[ord[n]]) * kDpar * kLog2e);
        gt[4 * p + h] = static_cast<float>(s * v.bvecs[3 * ord[n]]);
        gt[4 * p + 2 + h] = static_cast<float>(s * v.bvecs[3 * ord[n] + 1]);
        gt[2 * NPg + n] = static_cast<float>(s * v.bvecs[3 * ord[n] + 2]);
      }
    }
    tab += v.n_meas;
    gr.table2_off = static_cast<int32_t>(h->tab2_pairs);
    h->tab2_pairs += ((v.n_meas + 3) & ~3) / 2;
    gr.gp_off = static_cast<int32_t>(gp);
    h->gp_layout[4 * g + 0] = gp;
    h->gp_layout[4 * g + 1] = gp + 4;
    h->gp_layout[4 * g + 2] = gp + 4 + gr.N4;
    h->gp_layout[4 * g + 3] = gp + 4 + 2 * gr.N4;
    gp += 4 + 2 * gr.N4 + kNGrid;
    h->yhat_off[g] = yh;
    yh += static_cast<int64_t>(gr.n_vox) * v.n_meas;
    Nmax = std::max(Nmax, v.n_meas);
    gr.tile0 = static_cast<int32_t>(h->tiles.size());
    const int px = (v.nx + P - 1) / P, py = (v.ny + P - 1) / P, pz = (v.nz + P - 1) / P;
    const int64_t npatch = static_cast<int64_t>(px) * py * pz;
    // pass 1 (parallel): masked voxels per patch
    std::vector<int32_t> pcount(npatch, 0);
    auto patch_box = [&](int64_t pi, int lo[3], int hi[3]) {
      const int a = static_cast<int>(pi / (static_cast<int64_t>(py) * pz)), b = static_cast<int>((pi / pz) % py),
                c3 = static_cast<int>(pi % pz);
      lo[0] = a * P, lo[1] = b * P, lo[2] = c3 * P;
      hi[0] = std::min(v.nx, (a + 1) * P), hi[1] = std::min(v.ny, (b + 1) * P), hi[2] = std::min(v.nz, (c3 + 1) * P);
    };
    parallel_chunks(npatch, 16, [&](int64_t b0, int64_t e0) {
      for (int64_t pi = b0; pi < e0; ++pi) {
        int lo[3], hi[3];
        patch_box(pi, lo, hi);
        int32_t n = 0;
        for (int x = lo[0]; x < hi[0]; ++x)
          for (int y = lo[1]; y < hi[1]; ++y)
            for (int z = lo[2]; z < hi[2]; ++z) n += vidx[g][(static_cast<int64_t>(x) * v.ny + y) * v.nz + z] >= 0;
        pcount[pi] = n;
      }
    });
    // tiles and patches in patch order (sequential, one entry per tile)
    std::vector<int32_t> ptile(npatch, -1);
    for (int64_t pi = 0; pi < npatch; ++pi) {
      if (pcount[pi] == 0) continue;
      const int pid = static_cast<int>(h->patches.size());
      const int tb = static_cast<int>(h->tiles.size());
      ptile[pi] = tb;
      for (int32_t s0 = 0; s0 < pcount[pi]; s0 += TV) {
        Tile t{};
        t.group = g;
        t.patch = pid;
        t.slot0 = static_cast<int32_t>(h->tiles.size()) * TV;
        t.count = std::min(TV, pcount[pi] - s0);
        t.y_off = yoff;
        t.ab_off = static_cast<int32_t>(aboff);
        t.n_meas = v.n_meas;
        yoff += static_cast<int64_t>((v.n_meas + 3) & ~3) * TV;
        aboff += 2 * v.n_meas;
        h->tiles.push_back(t);
      }
      h->patches.push_back({tb, static_cast<int>(h->tiles.size())});
    }
    // pass 2 (parallel): the slots of each patch's voxels, in C order within the patch; grid
    // positions outside the mask (the patch boxes cover the grid) get slot -1
    parallel_chunks(npatch, 16, [&](int64_t b0, int64_t e0) {
      for (int64_t pi = b0; pi < e0; ++pi) {
        int lo[3], hi[3];
        patch_box(pi, lo, hi);
        int slot = ptile[pi] * TV;
        for (int x = lo[0]; x < hi[0]; ++x)
          for (int y = lo[1]; y < hi[1]; ++y)
            for (int z = lo[2]; z < hi[2]; ++z) {
              const int64_t gi = (static_cast<int64_t>(x) * v.ny + y) * v.nz + z;
              const int32_t vi = vidx[g][gi];
              if (vi < 0) {
                pl.slot_of_grid[gr.grid_off + gi] = -1;
                continue;
              }
              const int64_t vg = h->vox0[g] + vi;
              pl.slot_of_vox[vg] = slot;
              pl.slot_of_grid[gr.grid_off + gi] = slot;
              pl.row_off[vg] = h->yhat_off[g] + static_cast<int64_t>(vi) * v.n_meas;
              ++slot;
            }
      }
    });
    gr.ntiles = static_cast<int32_t>(h->tiles.size()) - gr.tile0;
  }
  h->ntiles = static_cast<int>(h->tiles.size());
  if (static_cast<int64_t>(h->ntiles) * TV > (1LL << 31) - 1) return fail(PRISM_E_SHAPE, "too many voxels");
  h->Vpad = h->ntiles * TV;
  h->Nmax = (Nmax + 3) & ~3;   // rows of the shared-memory table (paired tables pad to 4)
  h->GP = gp;
  h->gp_layout[4 * static_cast<size_t>(n_vols)] = gp;
  h->ypack_len = yoff;
  h->ab_len = aboff;
  h->tab_rows = tab;
  h->yhat_off[n_vols] = yh;
  h->yhat_len = yh;
  // the per-slot tables (mask-order index, coordinates, neighbour slots and flags) are built
  // on the device from slot_of_grid (launch_slot_data)
  return PRISM_OK;
}

template <typename T, typename A>
int upload(T* dst, const std::vector<T, A>& src, cudaStream_t st) {
  if (src.empty()) return PRISM_OK;
  CK(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return PRISM_OK;
}

#define RC(x)                    \
  do {                           \
    int r_ = (x);                \
    if (r_ != PRISM_OK) return r_; \
  } while (0)

int init_impl(prism_handle* h, const prism_volume* vols, int n_vols, const std::vector<int64_t>& counts,
              cudaStream_t st) {
  const prism_options& o = h->opt;
  h->K = o.K;
  h->Q = 4 * o.K + 5;
  h->XF = 4 * o.K + 3;
  h->cal = o.calibration != 0;
  h->nb = (o.lam_sp > 0.f) || (o.lam_dir > 0.f);
  h->ks = &kernels_for_k(o.K);
  h->TV = h->NT / h->TPV;
  // Host signals start their copy to the device before the plan is built: a copy needs only the
  // voxel count, and the DMA then runs while the host builds the plan. All copies start at once
  // when together they take at most a quarter of the free device memory; otherwise each volume
  // is copied in turn below.
  std::vector<float*> early(n_vols, nullptr);
  {
    size_t bytes = 0;
    for (int g = 0; g < n_vols; ++g)
      if (vols[g].mem == PRISM_MEM_HOST) bytes += sizeof(float) * static_cast<size_t>(counts[g]) * vols[g].n_meas;
    size_t fr = 0, tot = 0;
    if (bytes > 0 && cudaMemGetInfo(&fr, &tot) == cudaSuccess && bytes <= fr / 4) {
      for (int g = 0; g < n_vols; ++g) {
        if (vols[g].mem != PRISM_MEM_HOST) continue;
        const size_t n = static_cast<size_t>(counts[g]) * vols[g].n_meas;
        RC(h->alloc(&early[g], n));
        CK(cudaMemcpyAsync(early[g], vols[g].signal, sizeof(float) * n, cudaMemcpyHostToDevice, st));
      }
    }
  }
  Plan pl;
  RC(build_plan(h, vols, n_vols, pl));
  const int Vp = h->Vpad, Q = h->Q, G = h->G;
  // group reduction geometry
  h->max_e = 3 + (h->cal ? 2 * h->Nmax : 0);
  std::vector<int32_t> split_off(G);
  int tot_split = 0;
  h->max_split = 1;
  for (int g = 0; g < G; ++g) {
    const int ns = (h->groups[g].ntiles + kSplitTiles - 1) / kSplitTiles;
    split_off[g] = tot_split;
    tot_split += ns;
    h->max_split = std::max(h->max_split, ns);
  }
  const int nce = (h->max_e + 255) / 256;
  // allocations
  RC(h->alloc(&h->d_tiles, h->ntiles));
  RC(h->alloc(&h->d_tile_order, h->ntiles));
  RC(h->alloc(&h->d_groups, G));
  RC(h->alloc(&h->d_y, h->ypack_len));
  RC(h->alloc(&h->d_theta, static_cast<size_t>(Q) * Vp));
  RC(h->alloc(&h->d_m, static_cast<size_t>(Q) * Vp));
  RC(h->alloc(&h->d_v, static_cast<size_t>(Q) * Vp));
  RC(h->alloc(&h->d_xf, 2 * static_cast<size_t>(h->XF) * Vp));
  RC(h->alloc(&h->d_hsp, static_cast<size_t>(h->K + 3) * Vp));
  RC(h->alloc(&h->d_lp, Vp));
  const size_t pg_len = (h->nb && o.fused) ? static_cast<size_t>(4 * h->K + 4) * Vp : 1;
  RC(h->alloc(&h->d_pg, pg_len));
  CK(cudaMemsetAsync(h->d_pg, 0, sizeof(float) * pg_len, st));
  RC(h->alloc(&h->d_gU, Vp));
  RC(h->alloc(&h->d_tile_ab, h->ab_len));
  RC(h->alloc(&h->d_tile_red, 4 * static_cast<size_t>(h->ntiles)));
  RC(h->alloc(&h->d_nbr, static_cast<size_t>(o.connectivity) * Vp));
  RC(h->alloc(&h->d_vcoord, Vp));
  RC(h->alloc(&h->d_vflag, Vp));
  RC(h->alloc(&h->d_table, h->tab_rows));
  RC(h->alloc(&h->d_table2, h->tab2_pairs));
  CK(cudaMemsetAsync(h->d_table2, 0, sizeof(MeasPair) * h->tab2_pairs, st));
  RC(h->alloc(&h->d_gtab, h->gtab.size()));
  RC(h->alloc(&h->d_runs, h->runs.size()));
  RC(h->alloc(&h->d_gparams, h->GP));
  RC(h->alloc(&h->d_gm, h->GP));
  RC(h->alloc(&h->d_gv, h->GP));
  RC(h->alloc(&h->d_gred, h->GP));
  RC(h->alloc(&h->d_gloss, G));
  RC(h->alloc(&h->d_gprior, G));
  RC(h->alloc(&h->d_hist, static_cast<size_t>(kHistLen) * G));
  RC(h->alloc(&h->d_queue, 4));
  RC(h->alloc(&h->d_done, 1));
  RC(h->alloc(&h->d_step, 1));
  RC(h->alloc(&h->d_status, 1));
  RC(h->alloc(&h->d_adamc, 2));
  RC(h->alloc(&h->d_slot_of_vox, h->V));
  RC(h->alloc(&h->d_vox_of_slot, Vp));
  RC(h->alloc(&h->d_slot_of_grid, pl.slot_of_grid.size()));
  RC(h->alloc(&h->d_row_off, h->V));
  RC(h->alloc(&h->d_order, std::max<int64_t>(h->tab_rows, 1)));
  RC(h->alloc(&h->d_split_off, G));
  RC(h->alloc(&h->d_part2, static_cast<size_t>(tot_split) * h->max_e));
  RC(h->alloc(&h->d_counters, static_cast<size_t>(G) * nce));
  RC(h->alloc(&h->d_gdone, 1));
  CK(cudaMemsetAsync(h->d_gdone, 0, sizeof(int32_t), st));
  if (h->cal) {
    // per group [nx][ny][8] then [nx][8][8] doubles for the separable bias-field adjoint
    std::vector<int64_t> bs(2 * static_cast<size_t>(G));
    int64_t tot = 0;
    for (int g = 0; g < G; ++g) {
      const GroupDev& gr = h->groups[g];
      bs[2 * g] = tot;
      tot += static_cast<int64_t>(gr.nx) * gr.ny * kGrid;
      bs[2 * g + 1] = tot;
      tot += static_cast<int64_t>(gr.nx) * kGrid * kGrid;
      h->max_nx = std::max(h->max_nx, gr.nx);
      h->max_ny = std::max(h->max_ny, gr.ny);
    }
    RC(h->alloc(&h->d_bscratch, tot));
    RC(h->alloc(&h->d_bs_off, 2 * static_cast<size_t>(G)));
    RC(upload(h->d_bs_off, bs, st));
  }
  if (!o.fused) {
    RC(h->alloc(&h->d_yhat, h->ypack_len));
    RC(h->alloc(&h->d_r, h->ypack_len));
  }
  RC(h->alloc(&h->d_grad, static_cast<size_t>(Q) * Vp));
  // zero state
  CK(cudaMemsetAsync(h->d_theta, 0, sizeof(float) * Q * static_cast<size_t>(Vp), st));
  CK(cudaMemsetAsync(h->d_m, 0, sizeof(float) * Q * static_cast<size_t>(Vp), st));
  CK(cudaMemsetAsync(h->d_v, 0, sizeof(float) * Q * static_cast<size_t>(Vp), st));
  CK(cudaMemsetAsync(h->d_xf, 0, sizeof(float) * 2 * h->XF * static_cast<size_t>(Vp), st));
  CK(cudaMemsetAsync(h->d_hsp, 0, sizeof(float) * (h->K + 3) * static_cast<size_t>(Vp), st));
  CK(cudaMemsetAsync(h->d_lp, 0, sizeof(float) * Vp, st));
  CK(cudaMemsetAsync(h->d_gU, 0, sizeof(float) * Vp, st));
  CK(cudaMemsetAsync(h->d_tile_ab, 0, sizeof(float) * std::max<int64_t>(h->ab_len, 1), st));
  CK(cudaMemsetAsync(h->d_tile_red, 0, sizeof(double) * 4 * h->ntiles, st));
  CK(cudaMemsetAsync(h->d_gparams, 0, sizeof(float) * h->GP, st));
  CK(cudaMemsetAsync(h->d_gm, 0, sizeof(float) * h->GP, st));
  CK(cudaMemsetAsync(h->d_gv, 0, sizeof(float) * h->GP, st));
  CK(cudaMemsetAsync(h->d_gred, 0, sizeof(double) * h->GP, st));
  CK(cudaMemsetAsync(h->d_gloss, 0, sizeof(double) * G, st));
  CK(cudaMemsetAsync(h->d_gprior, 0, sizeof(double) * G, st));
  CK(cudaMemsetAsync(h->d_hist, 0, sizeof(double) * kHistLen * G, st));
  CK(cudaMemsetAsync(h->d_queue, 0, sizeof(int32_t) * 4, st));
  CK(cudaMemsetAsync(h->d_done, 0, sizeof(int32_t), st));
  CK(cudaMemsetAsync(h->d_step, 0, sizeof(int32_t), st));
  CK(cudaMemsetAsync(h->d_status, 0, sizeof(int32_t), st));
  CK(cudaMemsetAsync(h->d_counters, 0, sizeof(int32_t) * G * nce, st));
  CK(cudaMemsetAsync(h->d_grad, 0, sizeof(float) * Q * static_cast<size_t>(Vp), st));
  // metadata
  RC(upload(h->d_tiles, h->tiles, st));
  RC(upload(h->d_tile_order, tile_queue_order(h->tiles, h->TV), st));
  RC(upload(h->d_groups, h->groups, st));
  RC(upload(h->d_slot_of_vox, pl.slot_of_vox, st));
  RC(upload(h->d_slot_of_grid, pl.slot_of_grid, st));
  CK(launch_slot_data(h->d_tiles, h->d_groups, h->G, h->groups.data(), h->d_slot_of_grid, h->d_slot_of_vox, h->V,
                      Vp, h->TV, h->opt.connectivity, h->d_vox_of_slot, h->d_vcoord, h->d_vflag, h->d_nbr, st));
  RC(upload(h->d_row_off, pl.row_off, st));
  RC(upload(h->d_order, h->order, st));
  RC(upload(h->d_gtab, h->gtab, st));
  RC(upload(h->d_runs, h->runs, st));
  RC(upload(h->d_split_off, split_off, st));
  fill_args(h);
  // per volume: b0 statistics, packing, table, sigma, parameters
  int* d_bad = nullptr;
  RC(h->alloc(&d_bad, 1));
  CK(cudaMemsetAsync(d_bad, 0, sizeof(int), st));
  for (int g = 0; g < G; ++g) {
    const prism_volume& v = vols[g];
    const GroupDev& gr = h->groups[g];
    const int N = v.n_meas;
    const int64_t Vg = gr.n_vox;
    const float* sig = v.signal;
    float* tmp_sig = early[g];
    if (tmp_sig) {
      sig = tmp_sig;
    } else if (v.mem == PRISM_MEM_HOST) {
      RC(h->alloc(&tmp_sig, static_cast<size_t>(Vg) * N));
      CK(cudaMemcpyAsync(tmp_sig, v.signal, sizeof(float) * Vg * N, cudaMemcpyHostToDevice, st));
      sig = tmp_sig;
    }
    std::vector<uint8_t> isb0(N);
    std::vector<float> bv(N), bvec(3 * N);   // in table order
    const int32_t* ord = h->order.data() + gr.table_off;
    for (int n = 0; n < N; ++n) {
      bv[n] = v.bvals[ord[n]];
      for (int c = 0; c < 3; ++c) bvec[3 * n + c] = v.bvecs[3 * ord[n] + c];
    }
    int nb0 = 0;
    for (int n = 0; n < N; ++n) {
      isb0[n] = v.bvals[n] <= 50.f;
      nb0 += isb0[n];
    }
    uint8_t* d_isb0 = nullptr;
    float *d_bv = nullptr, *d_bvec = nullptr, *d_b0 = nullptr;
    double* d_part = nullptr;
    const int nbk = static_cast<int>((Vg + 255) / 256);
    RC(h->alloc(&d_isb0, N));
    RC(h->alloc(&d_bv, N));
    RC(h->alloc(&d_bvec, 3 * N));
    RC(h->alloc(&d_b0, Vg));
    RC(h->alloc(&d_part, nbk));
    RC(upload(d_isb0, isb0, st));
    RC(upload(d_bv, bv, st));
    RC(upload(d_bvec, bvec, st));
    CK(launch_b0_stats(sig, Vg, N, d_isb0, nb0, d_b0, d_part, d_bad, st));
    CK(launch_sigma_init(d_part, nbk, Vg, nb0, o.sigma_init, h->d_gparams + gr.gp_off, st));
    CK(launch_pack(h->ia, sig, d_b0, h->d_vox_of_slot, h->d_order + gr.table_off, h->vox0[g], gr.tile0,
                   gr.tile0 + gr.ntiles, N, h->d_y, d_bad, st));
    CK(launch_table(d_bv, d_bvec, N, h->d_table + gr.table_off, st));
    CK(launch_pair_table(h->d_table + gr.table_off, N, h->d_table2 + gr.table2_off, st));
    if (v.init) {
      const float* in = v.init;
      float* tmp_in = nullptr;
      if (v.mem == PRISM_MEM_HOST) {
        RC(h->alloc(&tmp_in, static_cast<size_t>(Vg) * Q));
        CK(cudaMemcpyAsync(tmp_in, v.init, sizeof(float) * Vg * Q, cudaMemcpyHostToDevice, st));
        in = tmp_in;
      }
      CK(launch_scatter_params(in, h->d_slot_of_vox + h->vox0[g], Vg, Q, Vp, h->d_theta, st));
    } else {
      CK(launch_default_init(h->d_slot_of_vox + h->vox0[g], h->d_vcoord, v.ny, v.nz, Vg, h->K, Vp,
                             static_cast<uint64_t>(o.seed) * 1315423911ull + g, h->d_theta, st));
    }
    // free per-volume temporaries (after the work that reads them)
    CK(cudaStreamSynchronize(st));
    for (void* p : {static_cast<void*>(tmp_sig), static_cast<void*>(d_isb0), static_cast<void*>(d_bv),
                    static_cast<void*>(d_bvec), static_cast<void*>(d_b0), static_cast<void*>(d_part)}) {
      if (!p) continue;
      auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
      if (it != h->allocs.end()) h->allocs.erase(it);
      cudaFree(p);
    }
  }
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (bad > 0)
    return fail(PRISM_E_NONFINITE, std::to_string(bad) + " voxel(s) with a non-finite signal or a non-positive b0 mean");
  CK(h->ks->transform(h->ia, 0, h->ntiles, st));
  CK(launch_adam_constants(h->ia, st));
  // launch geometry of the fused kernel
  const int NW = h->NT / 32;
  h->shell = o.fused && !h->cal && o.loss == PRISM_LOSS_MSE && h->TPV == 1 && o.K <= 3 && h->shells_even &&
             o.shells == 0;
  const size_t ring = static_cast<size_t>(kStages) * kChunk * (kFusedThreads / h->TPV) * sizeof(float);
  if (h->shell) {
    h->fused_smem = 3 * static_cast<size_t>(h->Nmax) * sizeof(float) + kMaxRuns * sizeof(ShellRun) +
                    static_cast<size_t>(kShellCols) * kFusedThreads * sizeof(float) + ring;
  } else {
    h->fused_smem = static_cast<size_t>(h->Nmax) * sizeof(MeasRow) + ring +
                    (h->cal ? kNGrid * sizeof(float) + static_cast<size_t>(NW) * 2 * h->Nmax * sizeof(float) : 0);
  }
  h->adj_smem = h->cal ? static_cast<size_t>(NW) * 2 * h->Nmax * sizeof(float) : 0;
  if (o.fused) {
    int dev = 0, sms = 0, bps = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(h->ks->fused_occupancy(o.loss, h->cal ? 1 : 0, h->TPV, h->shell ? 1 : 0, h->NT, h->fused_smem, &bps));
    if (bps < 1) return fail(PRISM_E_CUDA, "fused kernel does not fit on an SM");
    h->fused_grid = std::max(1, std::min(h->ntiles, sms * bps));
  }
  CK(cudaStreamSynchronize(st));
  return PRISM_OK;
}

int choose_shape(const prism_options& o, int64_t V, bool shell, int* tpv, int* nt) {
  // Measured on GB300 (bundle phantoms, K = 3 and 5, MSE and NLL): sixteen lanes per voxel
  // below 2,048 voxels, four below 32,768 (1.1-1.9x faster than one). Above, one thread per
  // voxel, except where its 128-voxel tiles come to about one wave of the SMs' resident CTAs
  // (0.75-1.25 waves: the last tiles then run nearly alone); four lanes then balance the SMs
  // better (40^3: 7-19 % faster; calibrated, 14-19 %). Where the shell loop applies (`shell`:
  // it needs one thread per voxel) four lanes pay only above one wave: 40^3 (0.82 waves) 20 %
  // slower than the shell loop, 45^3 (1.17 waves) 2 % faster, 47^3 (1.33 waves) 4 % slower.
  if (o.threads_per_voxel) {
    *tpv = o.threads_per_voxel;
  } else if (V < 2048) {
    *tpv = 16;
  } else if (V < 32768) {
    *tpv = 4;
  } else {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 152;
    }
    // CTAs per SM of the one-thread-per-voxel kernel (3 for five fibers, NLL or calibration)
    const int occ = (o.K >= 5 || o.loss == PRISM_LOSS_NLL || o.calibration) ? 3 : 4;
    const double waves = static_cast<double>(V) / 128.0 / (static_cast<double>(sms) * occ);
    *tpv = (waves > (shell ? 1.0 : 0.75) && waves <= 1.25) ? 4 : 1;
  }
  // the fused kernel is compiled for 128-thread CTAs (4 resident per SM)
  *nt = o.fused ? 128 : (o.cta_threads ? o.cta_threads : 128);
  return PRISM_OK;
}

// Whether the fused kernel would take the shell loop with one thread per voxel: MSE without
// calibration, K <= 3, shells not switched off, and every volume's b-value shells (runs of
// equal b in sorted order) of even length and at most kMaxRuns of them.
bool shells_apply(const prism_volume* vols, int n, const prism_options& o) {
  if (!o.fused || o.loss != PRISM_LOSS_MSE || o.calibration || o.K > 3 || o.shells != 0) return false;
  for (int g = 0; g < n; ++g) {
    std::vector<float> b(vols[g].bvals, vols[g].bvals + vols[g].n_meas);
    std::sort(b.begin(), b.end());
    int runs = 0;
    for (size_t i = 0; i < b.size();) {
      size_t j = i + 1;
      while (j < b.size() && b[j] == b[i]) ++j;
      if ((j - i) % 2 != 0) return false;
      ++runs;
      i = j;
    }
    if (runs > kMaxRuns) return false;
  }
  return true;
}

// Masked voxels of each volume.
std::vector<int64_t> count_voxels(const prism_volume* vols, int n) {
  std::vector<int64_t> V(n, 0);
  for (int g = 0; g < n; ++g) {
    const int64_t ng = static_cast<int64_t>(vols[g].nx) * vols[g].ny * vols[g].nz;
    constexpr int64_t kChunkN = 1 << 18;
    const int64_t nch = (ng + kChunkN - 1) / kChunkN;
    std::vector<int64_t> cc(nch, 0);
    parallel_chunks(nch, 4, [&](int64_t b, int64_t e) {
      for (int64_t k = b; k < e; ++k) {
        int64_t c = 0;
        for (int64_t i = k * kChunkN; i < std::min(ng, (k + 1) * kChunkN); ++i) c += vols[g].mask[i] != 0;
        cc[k] = c;
      }
    });
    for (int64_t c : cc) V[g] += c;
  }
  return V;
}

int build_graphs(prism_handle* h) {
  CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  RC(capture_graph(h, 1, &h->g1));
  RC(capture_graph(h, kGraphUnroll, &h->gU));
  return PRISM_OK;
}

// A device buffer freed when it goes out of scope.
struct DevTmp {
  void* p = nullptr;
  DevTmp() = default;
  DevTmp(const DevTmp&) = delete;
  DevTmp& operator=(const DevTmp&) = delete;
  DevTmp(DevTmp&& o) noexcept : p(o.p) { o.p = nullptr; }
  ~DevTmp() {
    if (p) cudaFree(p);
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

int create_handle(const prism_volume* vols, int n_vols, const std::vector<int64_t>& counts, const prism_options& o,
                  int tpv, int nt, cudaStream_t st, prism_handle** out) {
  std::unique_ptr<prism_handle> h(new (std::nothrow) prism_handle());
  if (!h) return fail(PRISM_E_OOM, "host allocation failed");
  h->opt = o;
  h->TPV = tpv;
  h->NT = nt;
  RC(init_impl(h.get(), vols, n_vols, counts, st));
  if (o.fused && o.use_graph) RC(build_graphs(h.get()));
  *out = h.release();
  return PRISM_OK;
}

// Autotuning of the launch shape (prism_options.autotune): lanes per voxel (1, 4 or 16, or the
// forced value) and, with one lane, the shell loop or the per-measurement loop, each timed for a
// few fused iterations on the problem itself or, above kTuneVoxels, on a bounded sample of it:
// per volume its fullest patches in proportion to its voxels (whole patches, the volume's |M|
// as normaliser), about four waves of 128-voxel tiles of a GB300's resident CTAs. The voxels
// per tile (128 / lanes) and the ring depth are fixed by the compiled kernels.
constexpr int64_t kTuneVoxels = 4LL * 152 * 4 * 128;

struct TuneSample {
  std::vector<prism_volume> vols;
  std::vector<std::vector<uint8_t>> masks;
  std::vector<std::vector<float>> host_sig;
  std::vector<DevTmp> dev_sig, dev_rows;
  std::vector<int64_t> counts;
};

int tune_sample(const prism_volume* vols, int n_vols, const std::vector<int64_t>& counts, int P, int64_t budget,
                cudaStream_t st, TuneSample& S) {
  int64_t V = 0;
  for (int64_t c : counts) V += c;
  S.vols.assign(vols, vols + n_vols);
  S.masks.resize(n_vols);
  S.host_sig.resize(n_vols);
  S.dev_sig.resize(n_vols);
  S.dev_rows.resize(n_vols);
  S.counts.assign(n_vols, 0);
  for (int g = 0; g < n_vols; ++g) {
    const prism_volume& v = vols[g];
    const int64_t ng = static_cast<int64_t>(v.nx) * v.ny * v.nz;
    const int px = (v.nx + P - 1) / P, py = (v.ny + P - 1) / P, pz = (v.nz + P - 1) / P;
    std::vector<int32_t> pcount(static_cast<size_t>(px) * py * pz, 0);
    auto pid_of = [&](int64_t i) {
      const int x = static_cast<int>(i / (static_cast<int64_t>(v.ny) * v.nz)), y = static_cast<int>((i / v.nz) % v.ny),
                z = static_cast<int>(i % v.nz);
      return (static_cast<int64_t>(x / P) * py + y / P) * pz + z / P;
    };
    for (int64_t i = 0; i < ng; ++i)
      if (v.mask[i]) ++pcount[pid_of(i)];
    std::vector<int32_t> order(pcount.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int32_t>(i);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return pcount[a] > pcount[b]; });
    const int64_t quota = std::max<int64_t>(1, budget * counts[g] / std::max<int64_t>(V, 1));
    std::vector<uint8_t> keep(pcount.size(), 0);
    int64_t got = 0;
    for (int32_t p : order) {
      if (got >= quota || pcount[p] == 0) break;
      keep[p] = 1;
      got += pcount[p];
    }
    S.masks[g].assign(v.mask, v.mask + ng);
    std::vector<int64_t> rows;
    int64_t r = 0;
    for (int64_t i = 0; i < ng; ++i) {
      if (!v.mask[i]) continue;
      if (keep[pid_of(i)]) rows.push_back(r);
      else S.masks[g][i] = 0;
      ++r;
    }
    const int N = v.n_meas;
    const int64_t n = static_cast<int64_t>(rows.size());
    prism_volume& pv = S.vols[g];
    pv.mask = S.masks[g].data();
    pv.init = nullptr;
    pv.norm_count = v.norm_count > 0 ? v.norm_count : static_cast<int32_t>(counts[g]);
    S.counts[g] = n;
    if (v.mem == PRISM_MEM_HOST) {
      S.host_sig[g].resize(static_cast<size_t>(n) * N);
      for (int64_t i = 0; i < n; ++i)
        std::memcpy(S.host_sig[g].data() + i * N, v.signal + rows[i] * N, sizeof(float) * N);
      pv.signal = S.host_sig[g].data();
    } else {
      CK(cudaMalloc(&S.dev_rows[g].p, sizeof(int64_t) * n));
      CK(cudaMemcpyAsync(S.dev_rows[g].p, rows.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
      CK(cudaMalloc(&S.dev_sig[g].p, sizeof(float) * n * N));
      CK(launch_gather_rows(v.signal, S.dev_rows[g].as<int64_t>(), n, N, S.dev_sig[g].as<float>(), st));
      pv.signal = S.dev_sig[g].as<float>();
    }
  }
  CK(cudaStreamSynchronize(st));
  return PRISM_OK;
}

void autotune_shape(const prism_volume* vols, int n_vols, const std::vector<int64_t>& counts, const prism_options& o,
                    cudaStream_t st, int* tpv, int* shells) {
  int64_t V = 0;
  for (int64_t c : counts) V += c;
  TuneSample S;
  const prism_volume* tv = vols;
  const std::vector<int64_t>* tc = &counts;
  if (V > kTuneVoxels) {
    if (tune_sample(vols, n_vols, counts, o.patch_dim, kTuneVoxels, st, S) != PRISM_OK) {
      g_err.clear();
      return;
    }
    tv = S.vols.data();
    tc = &S.counts;
  }
  prism_options oc = o;
  oc.use_graph = 0;
  oc.autotune = 0;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return;
  }
  float best = 1e30f;
  const int lanes[3] = {1, 4, 16};
  for (int lane : lanes) {
    if (o.threads_per_voxel && lane != o.threads_per_voxel) continue;
    for (int sh : {0, -1}) {
      if (o.shells == -1 && sh == 0) continue;
      oc.shells = sh;
      prism_handle* hc = nullptr;
      if (create_handle(tv, n_vols, *tc, oc, lane, 128, st, &hc) != PRISM_OK) {
        g_err.clear();
        continue;
      }
      int rc = PRISM_OK;
      for (int i = 0; i < 2 && rc == PRISM_OK; ++i) rc = enqueue_fused_iter(hc, st);
      // the fastest of three rounds of four iterations (one round of a small batch is a
      // fraction of a millisecond, where a single round's noise can reorder candidates 10 %
      // apart)
      float ms = 1e30f;
      for (int round = 0; round < 3 && rc == PRISM_OK; ++round) {
        cudaEventRecord(e0, st);
        for (int i = 0; i < 4 && rc == PRISM_OK; ++i) rc = enqueue_fused_iter(hc, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float r = 0.f;
        cudaEventElapsedTime(&r, e0, e1);
        ms = std::min(ms, r);
      }
      const bool shell_used = hc->shell;
      delete hc;
      if (rc == PRISM_OK && ms < best) {
        best = ms;
        *tpv = lane;
        *shells = shell_used ? 0 : -1;
      }
      // the per-measurement loop is a second candidate only where the shell loop applied
      if (!shell_used) break;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  g_err.clear();
}

}  // namespace

extern "C" int prism_fit_init(const prism_volume* vols, int32_t n_vols, const prism_options* opt, void* stream,
                              prism_handle** out) {
  g_err.clear();
  if (!out) return fail(PRISM_E_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!vols || n_vols < 1) return fail(PRISM_E_INVALID_ARG, "at least one volume is required");
  prism_options o;
  if (opt) o = *opt;
  else prism_default_options(&o);
  RC(validate_options(o));
  for (int g = 0; g < n_vols; ++g) RC(validate_volume(vols[g], g));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const std::vector<int64_t> counts = count_voxels(vols, n_vols);
  int64_t V = 0;
  for (int64_t c : counts) V += c;
  int tpv = 1, nt = 128;
  choose_shape(o, V, shells_apply(vols, n_vols, o), &tpv, &nt);
  if (o.autotune && o.fused) {
    int shells = o.shells;
    autotune_shape(vols, n_vols, counts, o, st, &tpv, &shells);
    o.shells = shells;
  }
  prism_handle* h = nullptr;
  const int rc = create_handle(vols, n_vols, counts, o, tpv, nt, st, &h);
  if (rc != PRISM_OK) return rc;
  *out = h;
  return PRISM_OK;
}

extern "C" int prism_step(prism_handle* h, int32_t n_iters, void* stream) {
  if (!h) return fail(PRISM_E_INVALID_ARG, "handle is NULL");
  if (n_iters < 0) return fail(PRISM_E_INVALID_ARG, "n_iters must be >= 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  h->forward_done = false;
  if (h->opt.fused && h->gU) {
    int n = n_iters;
    while (n >= kGraphUnroll) {
      CK(cudaGraphLaunch(h->gU, st));
      n -= kGraphUnroll;
    }
    for (; n > 0; --n) CK(cudaGraphLaunch(h->g1, st));
  } else {
    for (int i = 0; i < n_iters; ++i) RC(h->opt.fused ? enqueue_fused_iter(h, st) : enqueue_plain_iter(h, st));
  }
  h->iters += n_iters;
  return PRISM_OK;
}

extern "C" int prism_sync(prism_handle* h, void* stream) {
  if (!h) return fail(PRISM_E_INVALID_ARG, "handle is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  int status = 0;
  CK(cudaMemcpy(&status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (status & kStTimeout) return fail(PRISM_E_TIMEOUT, "a bounded device wait (table bulk copy) timed out");
  if (status & kStNonfinite) return fail(PRISM_E_NONFINITE, "the objective became non-finite");
  return PRISM_OK;
}

extern "C" int prism_wait_probe(prism_handle* h, int32_t max_polls, void* stream) {
  if (!h) return fail(PRISM_E_INVALID_ARG, "handle is NULL");
  if (max_polls < 1 || max_polls > (1 << 20)) return fail(PRISM_E_INVALID_ARG, "max_polls must be in 1..1048576");
  CK(launch_wait_probe(h->d_status, max_polls, static_cast<cudaStream_t>(stream)));
  return PRISM_OK;
}

extern "C" int prism_info(const prism_handle* h, int64_t* n_vox, int32_t* n_groups, int32_t* q,
                          int64_t* n_group_params, int64_t* iterations) {
  if (!h) return fail(PRISM_E_INVALID_ARG, "handle is NULL");
  if (n_vox) *n_vox = h->V;
  if (n_groups) *n_groups = h->G;
  if (q) *q = h->Q;
  if (n_group_params) *n_group_params = h->GP;
  if (iterations) *iterations = h->iters;
  return PRISM_OK;
}

extern "C" int prism_get_shape(const prism_handle* h, int32_t* threads_per_voxel, int32_t* tile_voxels,
                               int32_t* fused_grid, int32_t* shell_loop) {
  if (!h) return fail(PRISM_E_INVALID_ARG, "handle is NULL");
  if (threads_per_voxel) *threads_per_voxel = h->TPV;
  if (tile_voxels) *tile_voxels = h->TV;
  if (fused_grid) *fused_grid = h->opt.fused ? h->fused_grid : 0;
  if (shell_loop) *shell_loop = h->shell ? 1 : 0;
  return PRISM_OK;
}

extern "C" int prism_get_params(prism_handle* h, float* out, int32_t mem, void* stream) {
  if (!h || !out) return fail(PRISM_E_INVALID_ARG, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n = static_cast<size_t>(h->V) * h->Q;
  if (mem == PRISM_MEM_DEVICE) {
    CK(launch_gather_params(h->d_theta, h->d_slot_of_vox, h->V, h->Q, h->Vpad, out, st));
    return PRISM_OK;
  }
  if (mem != PRISM_MEM_HOST) return fail(PRISM_E_INVALID_ARG, "mem must be HOST or DEVICE");
  float* tmp = nullptr;
  CK(cudaMalloc(&tmp, n * sizeof(float)));
  cudaError_t e = launch_gather_params(h->d_theta, h->d_slot_of_vox, h->V, h->Q, h->Vpad, tmp, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, n * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "prism_get_params");
  return PRISM_OK;
}

extern "C" int prism_set_params(prism_handle* h, const float* in, int32_t mem, void* stream) {
  if (!h || !in) return fail(PRISM_E_INVALID_ARG, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t n = static_cast<size_t>(h->V) * h->Q;
  const float* src = in;
  float* tmp = nullptr;
  if (mem == PRISM_MEM_HOST) {
    CK(cudaMalloc(&tmp, n * sizeof(float)));
    CK(cudaMemcpyAsync(tmp, in, n * sizeof(float), cudaMemcpyHostToDevice, st));
    src = tmp;
  } else if (mem != PRISM_MEM_DEVICE) {
    return fail(PRISM_E_INVALID_ARG, "mem must be HOST or DEVICE");
  }
  cudaError_t e = launch_scatter_params(src, h->d_slot_of_vox, h->V, h->Q, h->Vpad, h->d_theta, st);
  if (e == cudaSuccess) e = h->ks->transform(h->ia, 0, h->ntiles, st);
  if (tmp) {
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(tmp);
  }
  if (e != cudaSuccess) return cuda_fail(e, "prism_set_params");
  h->forward_done = false;
  return PRISM_OK;
}

extern "C" int prism_get_fibers(prism_handle* h, float* dirs, float* fracs, uint8_t* peaks, float rel_thresh,
                                int32_t mem, void* stream) {
  if (!h) return fail(PRISM_E_INVALID_ARG, "handle is NULL");
  if (!(rel_thresh >= 0.f && rel_thresh <= 1.f)) return fail(PRISM_E_INVALID_ARG, "rel_thresh must be in [0, 1]");
  if (mem != PRISM_MEM_HOST && mem != PRISM_MEM_DEVICE) return fail(PRISM_E_INVALID_ARG, "mem must be HOST or DEVICE");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int K = h->K;
  const size_t nd = static_cast<size_t>(h->V) * K * 3, nf = static_cast<size_t>(h->V) * (K + 3),
               np = static_cast<size_t>(h->V) * K;
  if (mem == PRISM_MEM_DEVICE) {
    CK(h->ks->fibers(h->ia, h->d_slot_of_vox, h->V, rel_thresh, dirs, fracs, peaks, st));
    return PRISM_OK;
  }
  char* tmp = nullptr;
  const size_t bytes = (dirs ? nd * 4 : 0) + (fracs ? nf * 4 : 0) + (peaks ? np : 0);
  CK(cudaMalloc(&tmp, bytes > 0 ? bytes : 1));
  float* dd = dirs ? reinterpret_cast<float*>(tmp) : nullptr;
  float* df = fracs ? reinterpret_cast<float*>(tmp + (dirs ? nd * 4 : 0)) : nullptr;
  uint8_t* dp = peaks ? reinterpret_cast<uint8_t*>(tmp + (dirs ? nd * 4 : 0) + (fracs ? nf * 4 : 0)) : nullptr;
  cudaError_t e = h->ks->fibers(h->ia, h->d_slot_of_vox, h->V, rel_thresh, dd, df, dp, st);
  if (e == cudaSuccess && dirs) e = cudaMemcpyAsync(dirs, dd, nd * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && fracs) e = cudaMemcpyAsync(fracs, df, nf * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && peaks) e = cudaMemcpyAsync(peaks, dp, np, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "prism_get_fibers");
  return PRISM_OK;
}

extern "C" int prism_group_layout(const prism_handle* h, int64_t* off) {
  if (!h || !off) return fail(PRISM_E_INVALID_ARG, "NULL argument");
  std::memcpy(off, h->gp_layout.data(), h->gp_layout.size() * sizeof(int64_t));
  return PRISM_OK;
}

extern "C" int prism_get_groups(prism_handle* h, float* out, int32_t mem, void* stream) {
  if (!h || !out) return fail(PRISM_E_INVALID_ARG, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const cudaMemcpyKind k = (mem == PRISM_MEM_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(out, h->d_gparams, h->GP * sizeof(float), k, st));
  if (mem == PRISM_MEM_HOST) CK(cudaStreamSynchronize(st));
  return PRISM_OK;
}

extern "C" int prism_set_groups(prism_handle* h, const float* in, int32_t mem, void* stream) {
  if (!h || !in) return fail(PRISM_E_INVALID_ARG, "NULL argument");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const cudaMemcpyKind k = (mem == PRISM_MEM_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(h->d_gparams, in, h->GP * sizeof(float), k, st));
  CK(launch_table_refresh(h->ga, h->ia, st));
  if (mem == PRISM_MEM_HOST) CK(cudaStreamSynchronize(st));
  h->forward_done = false;
  return PRISM_OK;
}

extern "C" int prism_get_loss(prism_handle* h, double* loss, double* hist, int32_t max_iters, int32_t* n_written) {
  if (!h) return fail(PRISM_E_INVALID_ARG, "handle is NULL");
  RC(prism_sync(h, nullptr));
  if (loss) CK(cudaMemcpy(loss, h->d_gloss, sizeof(double) * h->G, cudaMemcpyDeviceToHost));
  int32_t nw = 0;
  if (hist && max_iters > 0) {
    int step = 0;
    CK(cudaMemcpy(&step, h->d_step, sizeof(int), cudaMemcpyDeviceToHost));
    const int avail = std::min<int>(step, kHistLen);
    nw = std::min<int>(avail, max_iters);
    std::vector<double> ring(static_cast<size_t>(kHistLen) * h->G);
    CK(cudaMemcpy(ring.data(), h->d_hist, ring.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int i = 0; i < nw; ++i) {
      const int it = step - nw + i;
      std::memcpy(hist + static_cast<size_t>(i) * h->G, ring.data() + static_cast<size_t>(it % kHistLen) * h->G,
                  sizeof(double) * h->G);
    }
  }
  if (n_written) *n_written = nw;
  return PRISM_OK;
}

extern "C" int prism_forward(prism_handle* h, const float* theta, const float* groups, float* yhat, double* loss,
                             void* stream) {
  if (!h) return fail(PRISM_E_INVALID_ARG, "handle is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!h->d_yhat) RC(h->alloc(&h->d_yhat, h->ypack_len));
  if (!h->d_r) RC(h->alloc(&h->d_r, h->ypack_len));
  if (theta) CK(launch_scatter_params(theta, h->d_slot_of_vox, h->V, h->Q, h->Vpad, h->d_theta, st));
  if (groups) {
    CK(cudaMemcpyAsync(h->d_gparams, groups, h->GP * sizeof(float), cudaMemcpyDeviceToDevice, st));
    CK(launch_table_refresh(h->ga, h->ia, st));
  }
  const IterArgs& a = h->ia;
  PlainArgs p{h->d_yhat, h->d_r, h->d_grad, 0, h->ntiles, 1};
  const int cal = h->cal ? 1 : 0;
  CK(h->ks->transform(a, 0, h->ntiles, st));
  CK(h->ks->synth(a, p, cal, h->TPV, h->NT, st));
  CK(launch_loss(a, p, h->opt.loss, st));
  if (h->opt.lam_sp > 0.f) CK(h->ks->prior_prep(a, 0, h->ntiles, st));
  CK(h->ks->prior(a, p, st));
  CK(launch_group_reduce(a, h->ga, 1, st));
  CK(launch_group_adam(a, h->ga, 1, st));
  if (loss) CK(cudaMemcpyAsync(loss, h->d_gloss, sizeof(double) * h->G, cudaMemcpyDeviceToDevice, st));
  if (yhat) CK(launch_gather_yhat(h->d_yhat, a, h->d_vox_of_slot, h->d_row_off, h->d_order, yhat, st));
  h->forward_done = true;
  return PRISM_OK;
}

extern "C" int prism_backward(prism_handle* h, float* grad_theta, float* grad_groups, void* stream) {
  if (!h) return fail(PRISM_E_INVALID_ARG, "handle is NULL");
  if (!h->forward_done) return fail(PRISM_E_STATE, "prism_backward needs a preceding prism_forward");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const IterArgs& a = h->ia;
  PlainArgs p{h->d_yhat, h->d_r, h->d_grad, 0, h->ntiles, 2};
  const int cal = h->cal ? 1 : 0;
  CK(h->ks->adjoint(a, p, cal, h->TPV, h->NT, h->adj_smem, st));
  CK(h->ks->prior(a, p, st));
  if (h->cal) CK(launch_bias_grad(a, h->ga, st));
  CK(launch_group_reduce(a, h->ga, 2, st));
  GroupArgs ga = h->ga;
  ga.gexport = grad_groups;
  if (grad_groups) CK(launch_group_adam(a, ga, 4, st));
  if (grad_theta) CK(launch_gather_params(h->d_grad, h->d_slot_of_vox, h->V, h->Q, h->Vpad, grad_theta, st));
  return PRISM_OK;
}

extern "C" int prism_profile(prism_handle* h, int32_t n_iters, void* stream, float* ms_out) {
  if (!h || !ms_out || n_iters < 1) return fail(PRISM_E_INVALID_ARG, "NULL argument or n_iters < 1");
  if (!h->opt.fused) return fail(PRISM_E_STATE, "prism_profile times the fused path; the handle is plain");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const IterArgs& a = h->ia;
  cudaEvent_t ev[4];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  double acc[4] = {0, 0, 0, 0};
  int rc = PRISM_OK;
  for (int i = 0; i < n_iters && rc == PRISM_OK; ++i) {
    cudaError_t e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess && h->opt.lam_sp > 0.f) e = h->ks->prior_prep(a, 0, h->ntiles, st);
    if (e == cudaSuccess && h->nb) e = h->ks->prior_grad(a, 0, h->ntiles, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess)
      e = h->ks->fused(a, h->opt.loss, h->cal ? 1 : 0, h->TPV, h->shell ? 1 : 0, h->fused_grid, h->NT, h->fused_smem,
                       st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], st);
    if (e == cudaSuccess && h->cal) e = launch_bias_grad(a, h->ga, st);
    if (e == cudaSuccess && h->cal) e = launch_group_reduce(a, h->ga, 1 | 2, st);
    if (e == cudaSuccess && h->cal) e = launch_group_adam(a, h->ga, 1 | 2, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "prism_profile");
      break;
    }
    float t01 = 0, t12 = 0, t23 = 0, t03 = 0;
    cudaEventElapsedTime(&t01, ev[0], ev[1]);
    cudaEventElapsedTime(&t12, ev[1], ev[2]);
    cudaEventElapsedTime(&t23, ev[2], ev[3]);
    cudaEventElapsedTime(&t03, ev[0], ev[3]);
    acc[0] += t12;
    acc[1] += t01;
    acc[2] += t23;
    acc[3] += t03;
    h->iters += 1;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc != PRISM_OK) return rc;
  for (int k = 0; k < 4; ++k) ms_out[k] = static_cast<float>(acc[k] / n_iters);
  h->forward_done = false;
  return PRISM_OK;
}

namespace {
struct StateHeader {
  uint32_t magic, version;
  int32_t K, Q, G, step;
  int64_t V, GP;
};
}  // namespace

extern "C" int prism_state_size(const prism_handle* h, int64_t* bytes) {
  if (!h || !bytes) return fail(PRISM_E_INVALID_ARG, "NULL argument");
  *bytes = static_cast<int64_t>(sizeof(StateHeader)) + 3 * h->V * h->Q * 4 + 3 * h->GP * 4;
  return PRISM_OK;
}

extern "C" int prism_get_state(prism_handle* h, void* host_buf, int64_t bytes, void* stream) {
  int64_t need = 0;
  RC(prism_state_size(h, &need));
  if (!host_buf || bytes < need) return fail(PRISM_E_INVALID_ARG, "state buffer too small");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaStreamSynchronize(st));
  StateHeader hd{kStateMagic, 1, h->K, h->Q, h->G, 0, h->V, h->GP};
  CK(cudaMemcpy(&hd.step, h->d_step, sizeof(int), cudaMemcpyDeviceToHost));
  char* p = static_cast<char*>(host_buf);
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  const size_t nvq = static_cast<size_t>(h->V) * h->Q;
  float* tmp = nullptr;
  CK(cudaMalloc(&tmp, nvq * sizeof(float)));
  const float* srcs[3] = {h->d_theta, h->d_m, h->d_v};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    e = launch_gather_params(srcs[i], h->d_slot_of_vox, h->V, h->Q, h->Vpad, tmp, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p, tmp, nvq * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    p += nvq * sizeof(float);
  }
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "prism_get_state");
  const float* gsrc[3] = {h->d_gparams, h->d_gm, h->d_gv};
  for (int i = 0; i < 3; ++i) {
    CK(cudaMemcpy(p, gsrc[i], h->GP * sizeof(float), cudaMemcpyDeviceToHost));
    p += h->GP * sizeof(float);
  }
  return PRISM_OK;
}

extern "C" int prism_set_state(prism_handle* h, const void* host_buf, int64_t bytes, void* stream) {
  int64_t need = 0;
  RC(prism_state_size(h, &need));
  if (!host_buf || bytes < need) return fail(PRISM_E_INVALID_ARG, "state buffer too small");
  StateHeader hd;
  const char* p = static_cast<const char*>(host_buf);
  std::memcpy(&hd, p, sizeof(hd));
  if (hd.magic != kStateMagic || hd.version != 1 || hd.K != h->K || hd.Q != h->Q || hd.G != h->G || hd.V != h->V ||
      hd.GP != h->GP || hd.step < 0)
    return fail(PRISM_E_STATE, "checkpoint does not match this problem");
  p += sizeof(hd);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nvq = static_cast<size_t>(h->V) * h->Q;
  float* tmp = nullptr;
  CK(cudaMalloc(&tmp, nvq * sizeof(float)));
  float* dsts[3] = {h->d_theta, h->d_m, h->d_v};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
    e = cudaMemcpyAsync(tmp, p, nvq * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_scatter_params(tmp, h->d_slot_of_vox, h->V, h->Q, h->Vpad, dsts[i], st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    p += nvq * sizeof(float);
  }
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(e, "prism_set_state");
  float* gdst[3] = {h->d_gparams, h->d_gm, h->d_gv};
  for (int i = 0; i < 3; ++i) {
    CK(cudaMemcpy(gdst[i], p, h->GP * sizeof(float), cudaMemcpyHostToDevice));
    p += h->GP * sizeof(float);
  }
  CK(cudaMemcpy(h->d_step, &hd.step, sizeof(int), cudaMemcpyHostToDevice));
  CK(launch_adam_constants(h->ia, st));
  CK(launch_table_refresh(h->ga, h->ia, st));
  CK(h->ks->transform(h->ia, 0, h->ntiles, st));
  CK(cudaStreamSynchronize(st));
  h->iters = hd.step;
  h->forward_done = false;
  return PRISM_OK;
}

namespace {
// Device buffer released on scope exit (temporaries of the slab entry points).
}  // namespace

extern "C" int prism_fit_init_slabs(const prism_volume* vol, int32_t slab, int32_t overlap, const prism_options* opt,
                                    void* stream, prism_handle** out) {
  g_err.clear();
  if (!out) return fail(PRISM_E_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!vol) return fail(PRISM_E_INVALID_ARG, "vol is NULL");
  if (slab < 1 || overlap < 0 || 2 * overlap > slab)
    return fail(PRISM_E_INVALID_ARG, "need slab >= 1 and 0 <= overlap <= slab / 2");
  RC(validate_volume(*vol, 0));
  prism_options o;
  if (opt) o = *opt;
  else prism_default_options(&o);
  RC(validate_options(o));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nx = vol->nx, ny = vol->ny, nz = vol->nz, N = vol->n_meas, Q = 4 * o.K + 5;
  // slabs along the last axis, stride slab - overlap, the last one reaching the last slice
  std::vector<int> z0s, z1s;
  for (int z0 = 0;; z0 += slab - overlap) {
    z0s.push_back(z0);
    z1s.push_back(std::min(z0 + slab, nz));
    if (z1s.back() >= nz) break;
  }
  const int S = static_cast<int>(z0s.size());
  // the slabs holding each slice: za[z] always, zb[z] = za[z] + 1 in an overlap (else -1); with
  // stride slab - overlap >= overlap no slice lies in three slabs
  std::vector<int32_t> za(nz, -1), zb(nz, -1);
  for (int s = 0; s < S; ++s)
    for (int z = z0s[s]; z < z1s[s]; ++z) {
      if (zb[z] >= 0) return fail(PRISM_E_INVALID_ARG, "a slice lies in three slabs");
      (za[z] < 0 ? za[z] : zb[z]) = s;
    }
  // whole-volume mask order (C order) -> per-slab mask order (the same relative order), in two
  // passes over chunks of x (counts, then the entries at the chunks' offsets)
  std::vector<std::vector<int64_t>> rows(S);
  std::vector<std::vector<uint8_t>> sub(S);
  for (int s = 0; s < S; ++s) sub[s].assign(static_cast<size_t>(nx) * ny * (z1s[s] - z0s[s]), 0);
  const int nxc = std::min(nx, 64);
  std::vector<int64_t> cnt(static_cast<size_t>(nxc + 1) * (S + 1), 0);   // [chunk + 1][S + 1]
  auto xr = [&](int c, int& xa, int& xe) {
    xa = static_cast<int>(static_cast<int64_t>(nx) * c / nxc);
    xe = static_cast<int>(static_cast<int64_t>(nx) * (c + 1) / nxc);
  };
  parallel_chunks(nxc, 1, [&](int64_t cb, int64_t ce) {
    for (int c = static_cast<int>(cb); c < ce; ++c) {
      int xa, xe;
      xr(c, xa, xe);
      int64_t* k = cnt.data() + static_cast<size_t>(c + 1) * (S + 1);
      for (int x = xa; x < xe; ++x)
        for (int y = 0; y < ny; ++y) {
          const uint8_t* m = vol->mask + (static_cast<int64_t>(x) * ny + y) * nz;
          for (int z = 0; z < nz; ++z)
            if (m[z]) {
              ++k[S];
              ++k[za[z]];
              if (zb[z] >= 0) ++k[zb[z]];
            }
        }
    }
  });
  for (int c = 0; c < nxc; ++c)
    for (int s = 0; s <= S; ++s) cnt[static_cast<size_t>(c + 1) * (S + 1) + s] += cnt[static_cast<size_t>(c) * (S + 1) + s];
  const int64_t V = cnt[static_cast<size_t>(nxc) * (S + 1) + S];
  for (int s = 0; s < S; ++s) rows[s].resize(static_cast<size_t>(cnt[static_cast<size_t>(nxc) * (S + 1) + s]));
  std::vector<int64_t> src0(V), src1(V);
  std::vector<int32_t> slab0(V), slab1(V);
  std::vector<float> w1(V);
  parallel_chunks(nxc, 1, [&](int64_t cb, int64_t ce) {
    std::vector<int64_t> at(S + 1);
    for (int c = static_cast<int>(cb); c < ce; ++c) {
      int xa, xe;
      xr(c, xa, xe);
      for (int s = 0; s <= S; ++s) at[s] = cnt[static_cast<size_t>(c) * (S + 1) + s];
      for (int x = xa; x < xe; ++x)
        for (int y = 0; y < ny; ++y) {
          const uint8_t* m = vol->mask + (static_cast<int64_t>(x) * ny + y) * nz;
          for (int z = 0; z < nz; ++z) {
            if (!m[z]) continue;
            const int64_t v = at[S]++;
            const int first = za[z], second = zb[z];
            const int64_t i0 = at[first]++;
            rows[first][i0] = v;
            sub[first][(static_cast<size_t>(x) * ny + y) * (z1s[first] - z0s[first]) + (z - z0s[first])] = 1;
            int64_t i1 = -1;
            float wt = 0.f;
            if (second >= 0) {
              i1 = at[second]++;
              rows[second][i1] = v;
              sub[second][(static_cast<size_t>(x) * ny + y) * (z1s[second] - z0s[second]) + (z - z0s[second])] = 1;
              // linear ramp across the overlap of slabs first and second
              wt = (static_cast<float>(z - z0s[second]) + 0.5f) / static_cast<float>(z1s[first] - z0s[second]);
            }
            slab0[v] = first;
            src0[v] = i0;
            slab1[v] = second;
            src1[v] = i1;
            w1[v] = wt;
          }
        }
    }
  });
  if (V == 0) return fail(PRISM_E_SHAPE, "the mask is empty");
  // non-empty slabs become the handle's volumes; handle voxel = vox0[g] + index in the slab
  std::vector<int> gidx(S, -1);
  std::vector<int64_t> vox0;
  int G = 0;
  int64_t acc = 0;
  for (int s = 0; s < S; ++s)
    if (!rows[s].empty()) {
      gidx[s] = G++;
      vox0.push_back(acc);
      acc += static_cast<int64_t>(rows[s].size());
    }
  parallel_chunks(V, 1 << 15, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      src0[i] += vox0[gidx[slab0[i]]];
      if (src1[i] >= 0) src1[i] += vox0[gidx[slab1[i]]];
    }
  });
  // whole-volume signal (and initial parameters) on the device, then one gathered copy per slab
  DevTmp dsig, dinit, drows;
  const float* sig = vol->signal;
  const float* init = vol->init;
  if (vol->mem == PRISM_MEM_HOST) {
    CK(cudaMalloc(&dsig.p, sizeof(float) * V * N));
    CK(cudaMemcpyAsync(dsig.p, vol->signal, sizeof(float) * V * N, cudaMemcpyHostToDevice, st));
    sig = dsig.as<float>();
    if (init) {
      CK(cudaMalloc(&dinit.p, sizeof(float) * V * Q));
      CK(cudaMemcpyAsync(dinit.p, vol->init, sizeof(float) * V * Q, cudaMemcpyHostToDevice, st));
      init = dinit.as<float>();
    }
  }
  CK(cudaMalloc(&drows.p, sizeof(int64_t) * acc));
  std::vector<DevTmp> ssig(G), sinit(G);
  std::vector<prism_volume> vols(G);
  for (int s = 0; s < S; ++s) {
    const int g = gidx[s];
    if (g < 0) continue;
    const int64_t n = static_cast<int64_t>(rows[s].size());
    int64_t* dr = drows.as<int64_t>() + vox0[g];
    CK(cudaMemcpyAsync(dr, rows[s].data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
    CK(cudaMalloc(&ssig[g].p, sizeof(float) * n * N));
    CK(launch_gather_rows(sig, dr, n, N, ssig[g].as<float>(), st));
    if (init) {
      CK(cudaMalloc(&sinit[g].p, sizeof(float) * n * Q));
      CK(launch_gather_rows(init, dr, n, Q, sinit[g].as<float>(), st));
    }
    prism_volume& pv = vols[g];
    pv = *vol;
    pv.nz = z1s[s] - z0s[s];
    pv.mem = PRISM_MEM_DEVICE;
    pv.mask = sub[s].data();
    pv.signal = ssig[g].as<float>();
    pv.init = init ? sinit[g].as<float>() : nullptr;
  }
  CK(cudaStreamSynchronize(st));
  prism_handle* h = nullptr;
  RC(prism_fit_init(vols.data(), G, &o, stream, &h));
  CK(cudaStreamSynchronize(st));
  h->slabbed = true;
  h->st_src0 = std::move(src0);
  h->st_src1 = std::move(src1);
  h->st_w1 = std::move(w1);
  *out = h;
  return PRISM_OK;
}

extern "C" int prism_stitch_slabs(prism_handle* h, float* s0, float* fracs, float* fin, float* dirs, int32_t mem,
                                  void* stream) {
  if (!h) return fail(PRISM_E_INVALID_ARG, "handle is NULL");
  if (!h->slabbed) return fail(PRISM_E_STATE, "the handle was not made by prism_fit_init_slabs");
  if (mem != PRISM_MEM_HOST && mem != PRISM_MEM_DEVICE) return fail(PRISM_E_INVALID_ARG, "mem must be HOST or DEVICE");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t n = static_cast<int64_t>(h->st_src0.size());
  const int K = h->K;
  DevTmp d0, d1, dw, out;
  CK(cudaMalloc(&d0.p, sizeof(int64_t) * n));
  CK(cudaMalloc(&d1.p, sizeof(int64_t) * n));
  CK(cudaMalloc(&dw.p, sizeof(float) * n));
  CK(cudaMemcpyAsync(d0.p, h->st_src0.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(d1.p, h->st_src1.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dw.p, h->st_w1.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st));
  const size_t ns = n, nf = n * (K + 3), nd = n * K * 3;
  float *o_s0 = s0, *o_fr = fracs, *o_fin = fin, *o_d = dirs;
  if (mem == PRISM_MEM_HOST) {
    CK(cudaMalloc(&out.p, sizeof(float) * (2 * ns + nf + nd)));
    float* b = out.as<float>();
    o_s0 = s0 ? b : nullptr;
    o_fin = fin ? b + ns : nullptr;
    o_fr = fracs ? b + 2 * ns : nullptr;
    o_d = dirs ? b + 2 * ns + nf : nullptr;
  }
  CK(h->ks->stitch(h->ia, h->d_slot_of_vox, n, d0.as<int64_t>(), d1.as<int64_t>(), dw.as<float>(), o_s0, o_fr,
                   o_fin, o_d, st));
  if (mem == PRISM_MEM_HOST) {
    if (s0) CK(cudaMemcpyAsync(s0, o_s0, sizeof(float) * ns, cudaMemcpyDeviceToHost, st));
    if (fin) CK(cudaMemcpyAsync(fin, o_fin, sizeof(float) * ns, cudaMemcpyDeviceToHost, st));
    if (fracs) CK(cudaMemcpyAsync(fracs, o_fr, sizeof(float) * nf, cudaMemcpyDeviceToHost, st));
    if (dirs) CK(cudaMemcpyAsync(dirs, o_d, sizeof(float) * nd, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  return PRISM_OK;
}

extern "C" void prism_fit_destroy(prism_handle* h) { delete h; }

extern "C" int prism_fit(const prism_volume* vols, int32_t n_vols, const prism_options* opt, int32_t n_iters,
                         float* params_out, double* loss_out, int32_t out_mem, void* stream) {
  if (out_mem != PRISM_MEM_HOST && out_mem != PRISM_MEM_DEVICE) return fail(PRISM_E_INVALID_ARG, "out_mem must be HOST or DEVICE");
  prism_handle* h = nullptr;
  RC(prism_fit_init(vols, n_vols, opt, stream, &h));
  std::unique_ptr<prism_handle> guard(h);
  RC(prism_step(h, n_iters, stream));
  if (params_out) RC(prism_get_params(h, params_out, out_mem, stream));
  RC(prism_sync(h, stream));
  if (loss_out) {
    if (out_mem == PRISM_MEM_HOST) {
      RC(prism_get_loss(h, loss_out, nullptr, 0, nullptr));
    } else {
      CK(cudaMemcpyAsync(loss_out, h->d_gloss, sizeof(double) * h->G, cudaMemcpyDeviceToDevice,
                         static_cast<cudaStream_t>(stream)));
      CK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    }
  }
  return PRISM_OK;
}
