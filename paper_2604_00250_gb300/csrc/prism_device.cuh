// Device-side data structures and helpers of the PRISM fitting kernels (sm_103a).
//
// Notation follows the paper: S0, fractions f (softmax over [csf, gm, wm_1..wm_K,
// res]), fiber directions d_k, intra-axonal fraction f_in (Sec. 2.2), bias field
// B = exp(U), U = trilinear(b_lr) (Sec. 2.3), per-measurement exp(alpha_n), beta_n,
// noise sigma = exp(sigma_log).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bessel_fit.h"

namespace prism {

constexpr int kGrid = 8;          // bias control grid edge (Sec. 2.3 item 1)
constexpr int kNGrid = 512;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kHalfLog2Pi = 0.9189385332046727f;   // log(2 pi) / 2
constexpr float kNormEps2 = 1e-24f;                  // |v| clamp 1e-12, squared

// Device status word bits (read by prism_sync).
enum : int { kStTimeout = 1, kStNonfinite = 2 };

// One row of the per-measurement table (64 bytes, 16-byte aligned for the bulk copy).
// With c = d_k . g_n and x = c^2 the fiber terms of Eq. 5 are
//   e1 = exp(-b D_par x) = 2^(nkpar x),
//   p  = exp(-b (D_par x + D_perp (1 - x))) = 2^(nkperp + nkd x),
//   E_wm = f_in e1 + (1 - f_in) p,   dE_wm/dc = c (An f_in e1 + Bn (1 - f_in) p).
struct __align__(16) MeasRow {
  float gx, gy, gz, nkpar;       // g_n; -b D_par log2(e)
  float nkperp, nkd, ecsf, egm;  // -b D_perp log2(e); -b (D_par - D_perp) log2(e); E_csf, E_gm (Eq. 4)
  float eres, An, Bn, A;         // E_res; -2 b D_par; 2 b (D_perp - D_par); exp(alpha_n) (Eq. 6)
  float beta, pad0, pad1, pad2;  // beta_n
};

// Paired table: measurements 2p and 2p+1 field-interleaved, so that every field of the
// pair is one aligned float2 for packed (f32x2) arithmetic. Eight float4 per pair:
//   {gx, gy} {gz, nkpar} {nkperp, nkd} {ecsf, egm} {eres, An} {Bn, A} {beta, -} {-, -}
// with each name standing for the float2 (value at 2p, value at 2p+1); rows past N are zero.
struct __align__(16) MeasPair {
  float4 q[8];
};
// Field positions (MeasRow order) of e^alpha_n and beta_n in the paired table.
constexpr int kPairFieldA = 11, kPairFieldBeta = 12;

// One run of equal b-values in a group's table order (a shell), for the shell loop of the fused
// kernel (one thread per voxel, MSE, no calibration): measurement pairs [p0, p1) and the
// isotropic decays of Eq. 4 at this b. The fiber terms (Eq. 5) use the scaled cosine
// c' = s c = g' . d with s = sqrt(b D_par log2 e) and g' = s g (the shell loop's gradient table):
//   f_in e1 = 2^(log2 f_in - c'^2),   (1 - f_in) p = 2^(rho (log2 f_in - c'^2) + C0 - b D_perp log2 e)
// with rho = 1 - D_perp / D_par and C0 = log2(1 - f_in) - rho log2 f_in per voxel, and
//   dE_wm/dd = -2 ln(2) c' (f_in e1 + rho (1 - f_in) p) g'.
struct __align__(16) ShellRun {
  int32_t p0, p1, b0, pad;         // pairs [p0, p1); b0 = 1 for b = 0 (every E of Eqs. 4-5 is 1)
  float ecsf, egm, eres, nbperp;   // E_csf, E_gm, E_res; -b D_perp log2(e)
};
constexpr int kMaxRuns = 16;        // shells per group the shell loop takes
constexpr int kShellCols = 10;      // per-thread shared-memory column of the shell loop (floats)
constexpr float kRho = 1.f - 0.4f / 1.7f;   // 1 - D_perp / D_par (Eq. 5)

// Programmatic dependent launch: wait until the grids this one depends on have completed and
// their writes are visible (a no-op for a grid launched without the programmatic attribute),
// and let the dependent grid start launching.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
constexpr float kTwoLn2 = 1.3862943611198906f;   // 2 ln 2: d(2^(-x^2))/dx = -2 ln 2 x 2^(-x^2)

// A tile: up to TV voxels of one patch, processed by one CTA.
struct Tile {
  int32_t group, patch, slot0, count;
  int64_t y_off;     // float offset of the packed [N][TV] signal block
  int32_t ab_off;    // float offset of the tile's [2][N] alpha/beta gradient partials
  int32_t n_meas;
};

struct GroupDev {
  int32_t nx, ny, nz, N;
  int32_t tile0, ntiles;
  int32_t table_off;   // first MeasRow of the group
  int32_t gp_off;      // packed group params: sigma_log at gp_off, alpha at +4, beta at +4+N4, b_lr at +4+2 N4
  int32_t N4;          // N rounded up to a multiple of 4
  int32_t n_vox;
  float inv_M;         // 1 / |M_g|
  int32_t calib;       // calibration learned for this group
  int64_t grid_off;    // offset of the group's [nx][ny][nz] slot map
  int32_t table2_off;  // first MeasPair of the group
  int32_t nb0p;        // leading table pairs whose two measurements both have b = 0 (see meas_order)
  int32_t run_off;     // first ShellRun of the group (shell loop)
  int32_t n_runs;      // its shells
  int32_t gtab_off;    // float offset of the group's gradient table: [NP / 2][4] {g_x, g_y} pairs, then [NP] g_z
  int32_t pad_;
};

// Kernel arguments shared by the iteration kernels (passed by value).
struct IterArgs {
  int32_t Q, Vpad, TV, ntiles, Nmax, G;
  int32_t VW;              // voxels per warp slice of the packed signal (32 / threads per voxel)
  const Tile* tiles;
  const int32_t* tile_order;   // queue position -> tile (full tiles first, partial ones by size)
  const GroupDev* groups;
  const float* y;          // packed b0-normalised signal
  float* theta;            // [Q][Vpad]
  float* m;                // Adam first moments [Q][Vpad]
  float* v;                // Adam second moments [Q][Vpad]
  float* xf;               // [2][4K+3][Vpad] fractions and unit directions (ping-pong by step parity)
  float* hsp;              // [K+3][Vpad] rho'(u) / |N| of the Huber-Laplacian prior
  float* lp;               // [Vpad] Huber-Laplacian prior value per voxel
  float* pg;               // [4K+4][Vpad] neighbour priors for the fused kernel (k_prior_grad)
  const int32_t* nbr;      // [n_nbr][Vpad] same-patch masked neighbour slots or -1
  const uint32_t* vcoord;  // [Vpad] x | y << 10 | z << 20
  const uint32_t* vflag;   // [Vpad] bits 0-5 TV neighbours (+x,-x,+y,-y,+z,-z) masked; bits 8-12 |N(x)|
  const MeasRow* table;    // per-group measurement tables
  const MeasPair* table2;  // the same, paired (see MeasPair)
  const float* gtab;       // per group gradient directions in table order (shell loop; see GroupDev)
  const ShellRun* runs;    // per group shells in table order (shell loop)
  const float* gparams;    // packed group parameters
  float* gU;               // [Vpad] dJ/dU(x)
  float* tile_ab;          // per-tile [2][N] alpha / beta gradient partials
  double* tile_red;        // per-tile [4]: data loss, dJ/dsigma_log, prior loss, spare
  int32_t* queue;          // persistent work-queue counter
  int32_t* done;           // CTAs finished (last one resets the queue)
  const int32_t* step;     // iterations completed
  const float* adamc;      // Adam step constants of the coming iteration t: lr / (1 - b1^t), 1 / sqrt(1 - b2^t)
  int32_t* status;         // device status word
  float lam_rep, lam_sparse, tau, lam_sp, huber_delta, lam_dir, w_tv, tv_eps;
  float lr, beta1, beta2, eps;
  int32_t optimizer;       // 0 Adam, 1 Rprop (m = previous gradient, v = step size)
  float eta_minus, eta_plus, step_min, step_max;
  int32_t nb_priors;       // spatial or directional prior active
  int32_t n_nbr;           // 6 or 26
  float lam_orphan, inv_s_orphan, lam_order;
  // Group finalisation done by the fused kernel's last CTA when no group has calibration:
  // objective per group, its history, Adam on sigma_log (NLL), step counter.
  int32_t fold_groups, loss_mode, hist_len;
  // Host side: launch the iteration's neighbour-prior kernels and the fused kernel after them as
  // programmatic dependents (each starts while its predecessor finishes and waits on the device,
  // griddepcontrol, before it reads what the predecessor writes).
  int32_t pdl;
  float* gparams_rw;       // same array as gparams
  float* gm;               // group Adam moments (packed like gparams)
  float* gv;
  double* gloss;           // [G]
  double* hist;            // [hist_len][G]
};

// Packed signal layout: a tile's block holds TV / VW warp slices; slice w holds NP x VW
// floats (NP = N rounded up to a multiple of 4, padding rows zero), so one warp's data
// for consecutive measurements is one contiguous, 16-byte aligned run.
// Within a slice, measurements are pair-interleaved: (n, voxel lv) sits at
// ((n / 2) VW + lv) 2 + n % 2, so one voxel's two measurements of a pair are one float2.
__device__ __forceinline__ size_t ypos(const Tile& tl, int n, int vl, int VW) {
  const int w = vl / VW;
  const int NP = (tl.n_meas + 3) & ~3;
  return static_cast<size_t>(tl.y_off) + static_cast<size_t>(w) * NP * VW +
         (static_cast<size_t>(n >> 1) * VW + (vl - w * VW)) * 2 + (n & 1);
}

// Auxiliary arguments of the unfused (plain) kernels.
struct PlainArgs {
  float* yhat;             // packed like y
  float* r;                // packed like y: dL/dy_hat
  float* grad;             // [Q][Vpad] raw-parameter gradient
  int32_t tile_begin, tile_end;
  int32_t mode;            // k_prior: bit 0 loss, bit 1 gradient
};

// ---------------------------------------------------------------------------
// PTX helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2f_(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2f_(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcpf_(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Bulk (non-tensor) TMA copy global -> shared, completing on `bar`. Both addresses
// 16-byte aligned and `bytes` a multiple of 16 (the caller guarantees it).
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bulk prefetch of [p, p + bytes) into L2 (16-byte aligned address, size a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// Bounded wait on phase `parity`; false if it did not complete within `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit = 1 << 22) {
  const uint32_t addr = smem_u32(bar);
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// Parameter update: Adam (Kingma & Ba; the Table 2 comparator) or Rprop (Riedmiller &
// Braun 1993, the paper's solver): the step grows by eta_plus while the gradient keeps
// its sign and shrinks by eta_minus after a change (that step is skipped and the stored
// gradient zeroed), within [step_min, step_max]; the initial step is lr. Rprop keeps the
// previous gradient in m and the step in v (v == 0: not started).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void rprop_update(float& th, float& m, float& v, float g, float lr, float eta_minus,
                                             float eta_plus, float step_min, float step_max) {
  float step = (v == 0.f) ? lr : v;
  const float s = g * m;
  if (s > 0.f) {
    step = fminf(step * eta_plus, step_max);
  } else if (s < 0.f) {
    step = fmaxf(step * eta_minus, step_min);
    g = 0.f;
  }
  if (g > 0.f) th -= step;
  else if (g < 0.f) th += step;
  m = g;
  v = step;
}

// ---------------------------------------------------------------------------
// Scalar helpers.
// ---------------------------------------------------------------------------

// Huber rho and its derivative (transition delta).
__device__ __forceinline__ float huber_rho(float r, float dl) {
  const float a = fabsf(r);
  return a <= dl ? 0.5f * r * r : dl * (a - 0.5f * dl);
}
__device__ __forceinline__ float huber_drho(float r, float dl) {
  return fabsf(r) <= dl ? r : copysignf(dl, r);
}

// Q(z) = 1 - I1(z)/I0(z) and L(z) = log(exp(-z) I0(z)) for z >= 0, float32.
// Power series below PRISM_BESSEL_ZS, fitted smooth functions of ZS/z above. The two Horner
// chains of each branch share their argument, so they run as one packed f32x2 chain over the
// interleaved tables (each lane the same round-to-nearest multiply-add as the scalar chain; on
// GB300 the DiSCo1-shaped NLL fit's fused kernel 9 % faster).
template <bool WANT_L>
__device__ __forceinline__ void bessel_QL(float z, float& Q, float& L) {
  if (z < PRISM_BESSEL_ZS) {
    const float t = 0.25f * z * z;
    const float2 tt = make_float2(t, t);
    float2 s = k_bessel_s01[PRISM_BESSEL_NSER - 1];
#pragma unroll
    for (int k = PRISM_BESSEL_NSER - 2; k >= 0; --k) s = __ffma2_rn(s, tt, k_bessel_s01[k]);
    const float i0 = s.x, i1 = s.y;
    Q = 1.f - 0.5f * z * i1 * rcpf_(i0);   // i0 >= 1
    if (WANT_L) L = lg2f_(i0) * kLn2 - z;
  } else {
    const float x = PRISM_BESSEL_ZS * rcpf_(z);
    if (WANT_L) {
      const float2 xx = make_float2(x, x);
      float2 p = k_bessel_pba[PRISM_BESSEL_DEG];
#pragma unroll
      for (int k = PRISM_BESSEL_DEG - 1; k >= 0; --k) p = __ffma2_rn(p, xx, k_bessel_pba[k]);
      Q = p.x * x * (1.f / PRISM_BESSEL_ZS);
      L = (lg2f_(p.y) - 0.5f * lg2f_(z)) * kLn2 - kHalfLog2Pi;
    } else {
      float pb = k_bessel_pb[PRISM_BESSEL_DEG];
#pragma unroll
      for (int k = PRISM_BESSEL_DEG - 1; k >= 0; --k) pb = fmaf(pb, x, k_bessel_pb[k]);
      Q = pb * x * (1.f / PRISM_BESSEL_ZS);
    }
  }
}

// U(x) = trilinear upsampling of the 8^3 grid at voxel (i, j, k) of an n-grid,
// align_corners = False: u = clamp((i + .5) 8 / n - .5, 0, 7).
struct TriW {
  int base;       // flat index of corner (i0, j0, k0)
  float w[3];     // fractional parts per axis
};
__device__ __forceinline__ TriW tri_weights(int i, int j, int k, int nx, int ny, int nz) {
  TriW t;
  int idx[3];
  const int c[3] = {i, j, k};
  const int n[3] = {nx, ny, nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float u = (c[a] + 0.5f) * (8.f / n[a]) - 0.5f;
    u = fminf(fmaxf(u, 0.f), 7.f);
    int i0 = min(static_cast<int>(floorf(u)), 6);
    idx[a] = i0;
    t.w[a] = u - i0;
  }
  t.base = (idx[0] * kGrid + idx[1]) * kGrid + idx[2];
  return t;
}
__device__ __forceinline__ float tri_eval(const float* blr, const TriW& t) {
  float s = 0.f;
#pragma unroll
  for (int cx = 0; cx < 2; ++cx)
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cz = 0; cz < 2; ++cz) {
        const float w = (cx ? t.w[0] : 1.f - t.w[0]) * (cy ? t.w[1] : 1.f - t.w[1]) *
                        (cz ? t.w[2] : 1.f - t.w[2]);
        s = fmaf(w, blr[t.base + (cx * kGrid + cy) * kGrid + cz], s);
      }
  return s;
}

__device__ __forceinline__ void unpack_coord(uint32_t c, int& x, int& y, int& z) {
  x = c & 1023;
  y = (c >> 10) & 1023;
  z = (c >> 20) & 1023;
}

// Warp reductions (xor butterfly; every lane ends with the sum).
template <int FIRST, int LAST>
__device__ __forceinline__ float warp_sum_range(float x) {
#pragma unroll
  for (int o = FIRST; o <= LAST; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
// Reduce-scatter over each run of W consecutive lanes (W = 32: the whole warp): every lane
// holds G values v[0..G-1] (G = 2, 4 or 8, G <= W); on return each lane holds the run-wide sum
// of v[m] for m = the top log2 G bits of its index in the run, i.e. m = (lane % W) >> (log2 W -
// log2 G). Halving exchanges (xor W/2, W/4, ...) move half of the remaining values per stage,
// then an all-reduce over the low lane bits: log2 W shuffles of G - 1 + (log2 W - log2 G) values
// in all, instead of G log2 W for G separate all-reduces.
template <int G, int W = 32>
__device__ __forceinline__ float warp_scatter_sum(float (&v)[G]) {
  static_assert(G == 2 || G == 4 || G == 8, "G must be 2, 4 or 8");
  static_assert((W == 8 || W == 16 || W == 32) && G <= W, "W must be 8, 16 or 32 and at least G");
  constexpr int LG = (G == 2) ? 1 : (G == 4) ? 2 : 3;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int st = 0; st < LG; ++st) {
    const int o = (W / 2) >> st;
    const int half = G >> (st + 1);
    const bool hi = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float send = hi ? v[k] : v[k + half];
      const float keep = hi ? v[k + half] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  float x = v[0];
#pragma unroll
  for (int o = (W / 2) >> LG; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

__device__ __forceinline__ double warp_sum_d(double x) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

}  // namespace prism
