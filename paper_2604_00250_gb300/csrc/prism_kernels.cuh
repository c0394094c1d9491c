// Templated PRISM iteration kernels (K fibers, TPV threads per voxel, loss mode,
// calibration on/off). Included by one translation unit per K.
//
// The forward model, data terms and priors follow the paper (Sec. 2.2 Eqs. 3-5,
// Sec. 2.3 Eq. 6, Sec. 2.4, Sec. 2.5 Eqs. 8-9); the gradient is the hand-written
// adjoint of those equations; the update is Adam (the paper's Table 2 comparator).
#pragma once

#include "prism_device.cuh"

namespace prism {

enum : int { kLossMSE = 0, kLossNLL = 1 };

// Per-voxel transformed parameters (Sec. 2.2 "Per-voxel parameters", Sec. 2.5 constraints).
template <int K>
struct Vox {
  float S0, dS0;      // softplus(s), sigmoid(s)
  float f[K + 3];     // [csf, gm, wm_1..wm_K, res]
  float d[K][3];      // unit fiber directions
  float inrm[K];      // 1 / max(|v_k|, 1e-12)
  float fin, omf;     // f_intra, 1 - f_intra
};

template <int K>
__device__ __forceinline__ void load_theta(const float* __restrict__ theta, int Vp, int slot, bool act,
                                           float (&th)[4 * K + 5]) {
#pragma unroll
  for (int q = 0; q < 4 * K + 5; ++q) th[q] = act ? theta[static_cast<size_t>(q) * Vp + slot] : 0.f;
}

// Per-voxel transforms (Sec. 2.2 "Per-voxel parameters", Sec. 2.5 constraints), evaluated with
// special-function-unit approximations (2^x, log2, 1/x, 1/sqrt: relative error ~2^-22). Every
// kernel uses this one definition, so the neighbour-prior inputs written by any kernel are
// bitwise the ones the fused kernel would write.
__device__ __forceinline__ float fexp(float x) { return ex2f_(x * kLog2e); }
__device__ __forceinline__ float frcp(float x) { return rcpf_(x); }
__device__ __forceinline__ float fsoftplus(float s) {   // max(s,0) + log1p(e^{-|s|})
  const float e = fexp(-fabsf(s));
  const float l = (e < 1e-3f) ? e * fmaf(-0.5f, e, 1.f) : lg2f_(1.f + e) * kLn2;
  return fmaxf(s, 0.f) + l;
}
__device__ __forceinline__ float fsigmoid(float s) { return frcp(1.f + fexp(-s)); }

template <int K>
__device__ __forceinline__ void transform(const float (&th)[4 * K + 5], Vox<K>& P) {
  constexpr int NF = K + 3;
  P.S0 = fsoftplus(th[0]);
  P.dS0 = fsigmoid(th[0]);
  float mx = th[1];
#pragma unroll
  for (int i = 1; i < NF; ++i) mx = fmaxf(mx, th[1 + i]);
  float sum = 0.f;
#pragma unroll
  for (int i = 0; i < NF; ++i) {
    P.f[i] = fexp(th[1 + i] - mx);
    sum += P.f[i];
  }
  const float isum = frcp(sum);
#pragma unroll
  for (int i = 0; i < NF; ++i) P.f[i] *= isum;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float vx = th[K + 4 + 3 * k], vy = th[K + 5 + 3 * k], vz = th[K + 6 + 3 * k];
    const float in = rsqrtf(fmaxf(vx * vx + vy * vy + vz * vz, kNormEps2));
    P.inrm[k] = in;
    P.d[k][0] = vx * in;
    P.d[k][1] = vy * in;
    P.d[k][2] = vz * in;
  }
  P.fin = fsigmoid(th[4 * K + 4]);
  P.omf = 1.f - P.fin;
}

__device__ __forceinline__ float fsqrt(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Gradient w.r.t. transformed parameters -> raw parameters (adjoint of `transform`). With
// RAWU, gfin is already the derivative w.r.t. the raw u of f_intra = sigmoid(u).
template <int K, bool RAWU = false>
__device__ __forceinline__ void chain_raw(const Vox<K>& P, float gS0, const float (&gf)[K + 3],
                                          const float (&gd)[K][3], float gfin, float (&g)[4 * K + 5]) {
  constexpr int NF = K + 3;
  g[0] = gS0 * P.dS0;
  float dot = 0.f;
#pragma unroll
  for (int i = 0; i < NF; ++i) dot = fmaf(P.f[i], gf[i], dot);
#pragma unroll
  for (int i = 0; i < NF; ++i) g[1 + i] = P.f[i] * (gf[i] - dot);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float pd = gd[k][0] * P.d[k][0] + gd[k][1] * P.d[k][1] + gd[k][2] * P.d[k][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) g[K + 4 + 3 * k + c] = (gd[k][c] - pd * P.d[k][c]) * P.inrm[k];
  }
  g[4 * K + 4] = RAWU ? gfin : gfin * P.fin * P.omf;
}

// Writes the fractions and unit directions a neighbour needs (xf layout [4K+3][Vpad]).
template <int K>
__device__ __forceinline__ void store_xf(float* __restrict__ xf, int Vp, int slot, const Vox<K>& P) {
#pragma unroll
  for (int i = 0; i < K + 3; ++i) xf[static_cast<size_t>(i) * Vp + slot] = P.f[i];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) xf[static_cast<size_t>(K + 3 + 3 * k + c) * Vp + slot] = P.d[k][c];
}

// One neighbour x of the voxel at `slot` in the Huber-Laplacian (subtracts x's rho'(u)/|N|
// from hs) and the directional-continuity term (value and direction gradient). x < 0 (no
// neighbour) contributes nothing; its loads then read the voxel's own rows.
template <int K>
__device__ __forceinline__ void nbr_term(const IterArgs& a, const Vox<K>& P, int x, int slot, float inv_n,
                                         float wdir, const float* __restrict__ xf_cur, float (&hs)[K + 3],
                                         float& val, float (&gd)[K][3]) {
  constexpr int NF = K + 3;
  const int Vp = a.Vpad;
  const bool ok = x >= 0;
  const int xx = ok ? x : slot;
  if (a.lam_sp > 0.f) {
#pragma unroll
    for (int c = 0; c < NF; ++c) {
      const float h = a.hsp[static_cast<size_t>(c) * Vp + xx];
      hs[c] -= ok ? h : 0.f;
    }
  }
  if (a.lam_dir > 0.f) {
    const int nx_cnt = max(1, static_cast<int>((a.vflag[xx] >> 8) & 31));
    const float wgt = inv_n + 1.f / static_cast<float>(nx_cnt);
    const float wv = ok ? wdir * inv_n : 0.f;
    const float ws = ok ? -2.f * wdir * wgt : 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float dx[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) dx[q] = xf_cur[static_cast<size_t>(K + 3 + 3 * k + q) * Vp + xx];
      const float c = P.d[k][0] * dx[0] + P.d[k][1] * dx[1] + P.d[k][2] * dx[2];
      val = fmaf(wv, 1.f - c * c, val);
      const float sc = ws * c;
#pragma unroll
      for (int q = 0; q < 3; ++q) gd[k][q] = fmaf(sc, dx[q], gd[k][q]);
    }
  }
}

// The neighbour priors of Sec. 2.4 at one voxel: the Huber-Laplacian (from the precomputed
// rho'(u)/|N| of the voxel and its neighbours) and directional continuity (from the neighbours'
// directions; only P.d is read). Returns the value; adds the gradient to gf / gd.
template <int K>
__device__ __forceinline__ float nbr_priors(const IterArgs& a, const Vox<K>& P, int slot, float inv_M,
                                            const float* __restrict__ xf_cur, float (&gf)[K + 3],
                                            float (&gd)[K][3]) {
  constexpr int NF = K + 3;
  const int Vp = a.Vpad;
  float val = 0.f;
  const int ncnt = (a.vflag[slot] >> 8) & 31;
  if (ncnt > 0) {
    const float inv_n = 1.f / static_cast<float>(ncnt);
    const float wsp = a.lam_sp * inv_M, wdir = a.lam_dir * inv_M;
    float hs[NF];
    if (a.lam_sp > 0.f) {
      val += a.lp[slot];
#pragma unroll
      for (int c = 0; c < NF; ++c) hs[c] = a.hsp[static_cast<size_t>(c) * Vp + slot] * static_cast<float>(ncnt);
    }
    if (a.n_nbr == 6) {
      // face neighbours: every index first, then every neighbour's data (a missing
      // neighbour reads the voxel's own row with weight 0), so that the gathers overlap
      int xs[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) xs[e] = a.nbr[static_cast<size_t>(e) * Vp + slot];
#pragma unroll
      for (int e = 0; e < 6; ++e) nbr_term<K>(a, P, xs[e], slot, inv_n, wdir, xf_cur, hs, val, gd);
    } else {
      for (int e = 0; e < a.n_nbr; ++e)
        nbr_term<K>(a, P, a.nbr[static_cast<size_t>(e) * Vp + slot], slot, inv_n, wdir, xf_cur, hs, val, gd);
    }
    if (a.lam_sp > 0.f) {
#pragma unroll
      for (int c = 0; c < NF; ++c) gf[c] = fmaf(wsp, hs[c], gf[c]);
    }
  }
  return val;
}

// Rows of the precomputed neighbour priors (k_prior_grad): gradient w.r.t. the K + 3 fractions,
// then the 3K direction components, then the value.
template <int K>
constexpr int kPgRows = (K + 3) + 3 * K + 1;

// Priors of Sec. 2.4 at one voxel: value, and gradient added to gS0 / gf / gd (transformed
// space). Repulsion, sparsity, orphan-WM suppression and fiber ordering are local; the
// neighbour priors are evaluated here (PRE = false) or read as the rows k_prior_grad wrote for
// this iteration (PRE = true).
template <int K, bool PRE = false>
__device__ __forceinline__ float priors(const IterArgs& a, const Vox<K>& P, int slot, float inv_M,
                                        const float* __restrict__ xf_cur, float& gS0, float (&gf)[K + 3],
                                        float (&gd)[K][3]) {
  constexpr int NF = K + 3;
  const int Vp = a.Vpad;
  float val = 0.f;
  if (a.lam_rep > 0.f && K > 1) {
    const float w = a.lam_rep * inv_M;
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
      for (int j = i + 1; j < K; ++j) {
        const float c = P.d[i][0] * P.d[j][0] + P.d[i][1] * P.d[j][1] + P.d[i][2] * P.d[j][2];
        const float ac = fabsf(c);
        const float fi = P.f[2 + i], fj = P.f[2 + j];
        val = fmaf(w * fi * fj, ac, val);
        gf[2 + i] = fmaf(w * fj, ac, gf[2 + i]);
        gf[2 + j] = fmaf(w * fi, ac, gf[2 + j]);
        const float sg = (c > 0.f) ? w * fi * fj : ((c < 0.f) ? -w * fi * fj : 0.f);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          gd[i][q] = fmaf(sg, P.d[j][q], gd[i][q]);
          gd[j][q] = fmaf(sg, P.d[i][q], gd[j][q]);
        }
      }
  }
  if (a.lam_sparse > 0.f) {
    const float w = a.lam_sparse * inv_M;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (P.f[2 + k] < a.tau) {
        val = fmaf(w, P.f[2 + k], val);
        gf[2 + k] += w;
      }
  }
  if (a.lam_orphan > 0.f) {   // lam mean exp(-S0/s) sum_k f_wm,k
    const float w = a.lam_orphan * inv_M;
    const float e = ex2f_(-P.S0 * a.inv_s_orphan * kLog2e);
    float sf = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      sf += P.f[2 + k];
      gf[2 + k] = fmaf(w, e, gf[2 + k]);
    }
    val = fmaf(w * e, sf, val);
    gS0 = fmaf(-w * a.inv_s_orphan * e, sf, gS0);
  }
  if (a.lam_order > 0.f && K > 1) {   // lam mean sum_k max(0, f_k+1 - f_k)
    const float w = a.lam_order * inv_M;
#pragma unroll
    for (int k = 0; k + 1 < K; ++k) {
      const float dfk = P.f[3 + k] - P.f[2 + k];
      if (dfk > 0.f) {
        val = fmaf(w, dfk, val);
        gf[3 + k] += w;
        gf[2 + k] -= w;
      }
    }
  }
  if (a.nb_priors) {
    if constexpr (PRE) {
      const float* pg = a.pg + slot;
#pragma unroll
      for (int c = 0; c < NF; ++c) gf[c] += pg[static_cast<size_t>(c) * Vp];
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int q = 0; q < 3; ++q) gd[k][q] += pg[static_cast<size_t>(NF + 3 * k + q) * Vp];
      val += pg[static_cast<size_t>(NF + 3 * K) * Vp];
    } else {
      val += nbr_priors<K>(a, P, slot, inv_M, xf_cur, gf, gd);
    }
  }
  return val;
}

// Total-variation term of the upsampled bias field at voxel (x, y, z) (Sec. 2.4 "Calibration
// regularizers"; its form is not given there: sqrt((B(x+e) - B(x))^2 + eps) per axis):
// forward pairs inside the mask count once; returns the value and adds dTV/dU(x) to gU.
__device__ __forceinline__ float tv_term(const float* blr, int x, int y, int z, const GroupDev& gr,
                                         uint32_t fl, float B0, float w, float eps, float& gU) {
  float val = 0.f;
  const int off[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (fl & (1u << (2 * ax))) {   // x + e masked
      const TriW t = tri_weights(x + off[ax][0], y + off[ax][1], z + off[ax][2], gr.nx, gr.ny, gr.nz);
      const float B1 = expf(tri_eval(blr, t));
      const float dB = B1 - B0;
      const float sq = sqrtf(dB * dB + eps);
      val = fmaf(w, sq, val);
      gU = fmaf(-w * dB / sq, B0, gU);
    }
    if (fl & (2u << (2 * ax))) {   // x - e masked
      const TriW t = tri_weights(x - off[ax][0], y - off[ax][1], z - off[ax][2], gr.nx, gr.ny, gr.nz);
      const float Bm = expf(tri_eval(blr, t));
      const float dB = B0 - Bm;
      const float sq = sqrtf(dB * dB + eps);
      gU = fmaf(w * dB / sq, B0, gU);
    }
  }
  return val;
}

// Voxel-level gradient accumulators of the data term (unscaled), per thread:
// q = dJ/dS at each measurement; gwa_k = sum q e1_k, gwb_k = sum q p_k (so that
// dJ/df_wm,k and dJ/df_in follow after the loop), gd_k = sum q dE_k/dc g.
template <int K>
struct Acc {
  float gS0, gcsf, ggm, gres;
  float gwa[K], gwb[K];
  float gd[K][3];
  float l1, l2, l3;   // MSE: sum r^2 | NLL: sum (y-|yh|)^2, sum |y yh| Q, sum L
  float u;            // sum_n r A B S (= dJ/dU unscaled, calibration)
};

template <int K>
__device__ __forceinline__ void acc_zero(Acc<K>& A) {
  A.gS0 = A.gcsf = A.ggm = A.gres = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    A.gwa[k] = A.gwb[k] = 0.f;
    A.gd[k][0] = A.gd[k][1] = A.gd[k][2] = 0.f;
  }
  A.l1 = A.l2 = A.l3 = A.u = 0.f;
}

// Sum of the accumulators over a voxel's TPV lanes, which lie STRIDE lanes apart.
template <int K, int TPV, int STRIDE = 1>
__device__ __forceinline__ void acc_reduce_tpv(Acc<K>& A) {
  if constexpr (TPV > 1) {
    A.gS0 = warp_sum_range<STRIDE, STRIDE * TPV / 2>(A.gS0);
    A.gcsf = warp_sum_range<STRIDE, STRIDE * TPV / 2>(A.gcsf);
    A.ggm = warp_sum_range<STRIDE, STRIDE * TPV / 2>(A.ggm);
    A.gres = warp_sum_range<STRIDE, STRIDE * TPV / 2>(A.gres);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      A.gwa[k] = warp_sum_range<STRIDE, STRIDE * TPV / 2>(A.gwa[k]);
      A.gwb[k] = warp_sum_range<STRIDE, STRIDE * TPV / 2>(A.gwb[k]);
#pragma unroll
      for (int c = 0; c < 3; ++c) A.gd[k][c] = warp_sum_range<STRIDE, STRIDE * TPV / 2>(A.gd[k][c]);
    }
    A.l1 = warp_sum_range<STRIDE, STRIDE * TPV / 2>(A.l1);
    A.l2 = warp_sum_range<STRIDE, STRIDE * TPV / 2>(A.l2);
    A.l3 = warp_sum_range<STRIDE, STRIDE * TPV / 2>(A.l3);
    A.u = warp_sum_range<STRIDE, STRIDE * TPV / 2>(A.u);
  }
}

// One (voxel, measurement) pair: forward model (Eqs. 3-6), data-term derivative, and
// accumulation of the adjoint. With EXT_R the caller supplies dL/dy_hat (plain
// adjoint); rr_out returns dL/dy_hat (unscaled) and u_out the unscaled r A B S.
// `ffin` / `fomf` are f_wm,k f_in and f_wm,k (1 - f_in).
template <int K, int LOSS, bool CAL, bool EXT_R>
__device__ __forceinline__ void pair(const Vox<K>& P, const float (&ffin)[K], const float (&fomf)[K],
                                     const MeasRow& R, float yv, float B, float inv_s2, float r_ext, Acc<K>& A,
                                     float& rr_out, float& u_out) {
  float T = P.f[0] * R.ecsf;
  T = fmaf(P.f[1], R.egm, T);
  T = fmaf(P.f[K + 2], R.eres, T);
  float e1[K], p[K], c[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    c[k] = fmaf(P.d[k][0], R.gx, fmaf(P.d[k][1], R.gy, P.d[k][2] * R.gz));
    const float c2 = c[k] * c[k];
    e1[k] = ex2f_(R.nkpar * c2);
    p[k] = ex2f_(fmaf(R.nkd, c2, R.nkperp));
    T = fmaf(ffin[k], e1[k], fmaf(fomf[k], p[k], T));
  }
  const float S = P.S0 * T;
  float yh, AB = 1.f;
  if (CAL) {
    AB = R.A * B;
    yh = fmaf(AB, S, R.beta);
  } else {
    yh = S;
  }
  float rr;
  if (EXT_R) {
    rr = r_ext;
  } else if (LOSS == kLossMSE) {
    rr = yh - yv;
    A.l1 = fmaf(rr, rr, A.l1);
  } else {
    const float ay = fabsf(yh);
    const float sy = (yh >= 0.f) ? yv : -yv;
    float Qz, Lz;
    bessel_QL<true>(yv * ay * inv_s2, Qz, Lz);
    const float e = yv - ay;
    A.l1 = fmaf(e, e, A.l1);
    A.l2 = fmaf(yv * ay, Qz, A.l2);
    A.l3 += Lz;
    rr = fmaf(sy, Qz, yh - sy);      // y_hat - y R(z), R = I1/I0
  }
  rr_out = rr;
  const float q = CAL ? rr * AB : rr;   // dJ/dS (unscaled)
  if (CAL) {
    u_out = q * S;
    A.u += u_out;
  }
  A.gS0 = fmaf(q, T, A.gS0);
  A.gcsf = fmaf(q, R.ecsf, A.gcsf);
  A.ggm = fmaf(q, R.egm, A.ggm);
  A.gres = fmaf(q, R.eres, A.gres);
  const float anf = R.An * P.fin, bno = R.Bn * P.omf;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    A.gwa[k] = fmaf(q, e1[k], A.gwa[k]);
    A.gwb[k] = fmaf(q, p[k], A.gwb[k]);
    const float w = (q * c[k]) * fmaf(bno, p[k], anf * e1[k]);   // q dE_wm/dc
    A.gd[k][0] = fmaf(w, R.gx, A.gd[k][0]);
    A.gd[k][1] = fmaf(w, R.gy, A.gd[k][1]);
    A.gd[k][2] = fmaf(w, R.gz, A.gd[k][2]);
  }
}

template <int K>
__device__ __forceinline__ void fiber_weights(const Vox<K>& P, float (&ffin)[K], float (&fomf)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    ffin[k] = P.f[2 + k] * P.fin;
    fomf[k] = P.f[2 + k] * P.omf;
  }
}

// ---------------------------------------------------------------------------
// Packed path (one thread per voxel; MSE or NLL, with or without calibration): two
// measurements per step in f32x2 arithmetic. Voxel constants are held duplicated; accumulators
// are float2 and are folded after the loop. The residual is taken as y - y_hat (signs
// restored when folding).
// ---------------------------------------------------------------------------
template <int K>
struct VoxP {
  float2 fcsf, fgm, fres, nS0, fin, omf;
  float2 d[K][3];
  float2 ffin[K], fomf[K];
};

template <int K>
struct AccP {
  float2 gcsf, ggm, gres, l1;
  float2 gwa[K], gwb[K];
  float2 gd[K][3];
  float l2, l3;   // Rician NLL only: sum y |y_hat| Q, sum L
  float2 u;       // calibration only: sum q S (dJ/dU unscaled, negated)
};

__device__ __forceinline__ float2 dup2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 ex2_2(float2 v) { return make_float2(ex2f_(v.x), ex2f_(v.y)); }

template <int K>
__device__ __forceinline__ void voxp_init(const Vox<K>& P, VoxP<K>& D, AccP<K>& A) {
  D.fcsf = dup2(P.f[0]);
  D.fgm = dup2(P.f[1]);
  D.fres = dup2(P.f[K + 2]);
  D.nS0 = dup2(-P.S0);
  D.fin = dup2(P.fin);
  D.omf = dup2(P.omf);
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int c = 0; c < 3; ++c) D.d[k][c] = dup2(P.d[k][c]);
    D.ffin[k] = dup2(P.f[2 + k] * P.fin);
    D.fomf[k] = dup2(P.f[2 + k] * P.omf);
  }
  const float2 z = make_float2(0.f, 0.f);
  A.gcsf = A.ggm = A.gres = A.l1 = z;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    A.gwa[k] = A.gwb[k] = z;
    A.gd[k][0] = A.gd[k][1] = A.gd[k][2] = z;
  }
  A.l2 = A.l3 = 0.f;
  A.u = z;
}

// Rician NLL terms of one measurement (Eq. 9) for the packed path: adds (y - |y_hat|)^2 to l1,
// y |y_hat| Q(z) to l2 and L(z) to l3, and returns dL/dy_hat unscaled (y_hat - y R(z)); a
// lane with m = 0 (padding) adds nothing.
__device__ __forceinline__ float nll_lane(float yh, float yv, float inv_s2, float m, float& l1, float& l2,
                                          float& l3) {
  const float ay = fabsf(yh);
  const float sy = (yh >= 0.f) ? yv : -yv;
  float Qz, Lz;
  bessel_QL<true>(yv * ay * inv_s2, Qz, Lz);
  const float e = yv - ay;
  l1 = fmaf(m * e, e, l1);
  l2 = fmaf(m * yv * ay, Qz, l2);
  l3 = fmaf(m, Lz, l3);
  return m * fmaf(sy, Qz, yh - sy);
}

// One packed step over measurements (2p, 2p+1). With MASK, lanes whose msk is 0 add nothing.
// MSE: the data-term accumulators take r = y - y_hat. Rician NLL: they take -dL/dy_hat
// (unscaled), the same sign convention, and l1..l3 collect the objective's sums.
// With CAL the prediction is y_hat = e^alpha_n B S + beta_n (Eq. 6, B2 = B dup): the adjoint
// accumulators take q = r e^alpha_n B, A.u collects q S, and uo / ro return q S and r of the
// two measurements for the per-measurement alpha / beta partials.
template <int K, bool MASK, int LOSS = kLossMSE, bool CAL = false>
__device__ __forceinline__ void step2(const VoxP<K>& D, const MeasPair& R, float2 y, float2 msk, AccP<K>& A,
                                      float inv_s2 = 0.f, float2 B2 = float2{1.f, 1.f}, float2* uo = nullptr,
                                      float2* ro = nullptr) {
  const float4 q0 = R.q[0], q1 = R.q[1], q2 = R.q[2], q3 = R.q[3], q4 = R.q[4], q5 = R.q[5];
  const float2 gx = lo2(q0), gy = hi2(q0), gz = lo2(q1), nkpar = hi2(q1);
  const float2 nkperp = lo2(q2), nkd = hi2(q2), ecsf = lo2(q3), egm = hi2(q3);
  const float2 eres = lo2(q4), An = hi2(q4), Bn = lo2(q5);
  float2 T = __fmul2_rn(D.fcsf, ecsf);
  T = __ffma2_rn(D.fgm, egm, T);
  T = __ffma2_rn(D.fres, eres, T);
  float2 c[K], e1[K], p[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    c[k] = __ffma2_rn(D.d[k][0], gx, __ffma2_rn(D.d[k][1], gy, __fmul2_rn(D.d[k][2], gz)));
    const float2 c2 = __fmul2_rn(c[k], c[k]);
    e1[k] = ex2_2(__fmul2_rn(nkpar, c2));
    p[k] = ex2_2(__ffma2_rn(nkd, c2, nkperp));
    T = __ffma2_rn(D.ffin[k], e1[k], __ffma2_rn(D.fomf[k], p[k], T));
  }
  float2 r, q;
  if constexpr (CAL) {
    const float4 q6 = R.q[6];
    const float2 AB = __fmul2_rn(hi2(q5), B2);                        // e^alpha_n B
    const float2 S = __fmul2_rn(make_float2(-D.nS0.x, -D.nS0.y), T);
    const float2 yh = __ffma2_rn(AB, S, lo2(q6));                      // + beta_n
    if constexpr (LOSS == kLossMSE) {
      r = __ffma2_rn(make_float2(-1.f, -1.f), yh, y);                  // y - y_hat
      if (MASK) r = __fmul2_rn(r, msk);
      A.l1 = __ffma2_rn(r, r, A.l1);
    } else {
      r.x = -nll_lane(yh.x, y.x, inv_s2, MASK ? msk.x : 1.f, A.l1.x, A.l2, A.l3);
      r.y = -nll_lane(yh.y, y.y, inv_s2, MASK ? msk.y : 1.f, A.l1.y, A.l2, A.l3);
    }
    q = __fmul2_rn(r, AB);
    const float2 u = __fmul2_rn(q, S);
    A.u = __fadd2_rn(A.u, u);
    *uo = u;
    *ro = r;
  } else {
    if constexpr (LOSS == kLossMSE) {
      r = __ffma2_rn(D.nS0, T, y);   // y - y_hat
      if (MASK) r = __fmul2_rn(r, msk);
      A.l1 = __ffma2_rn(r, r, A.l1);
    } else {
      const float2 yh = __fmul2_rn(D.nS0, T);   // -y_hat
      r.x = -nll_lane(-yh.x, y.x, inv_s2, MASK ? msk.x : 1.f, A.l1.x, A.l2, A.l3);
      r.y = -nll_lane(-yh.y, y.y, inv_s2, MASK ? msk.y : 1.f, A.l1.y, A.l2, A.l3);
    }
    q = r;
  }
  A.gcsf = __ffma2_rn(q, ecsf, A.gcsf);
  A.ggm = __ffma2_rn(q, egm, A.ggm);
  A.gres = __ffma2_rn(q, eres, A.gres);
  const float2 anf = __fmul2_rn(An, D.fin), bno = __fmul2_rn(Bn, D.omf);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    A.gwa[k] = __ffma2_rn(q, e1[k], A.gwa[k]);
    A.gwb[k] = __ffma2_rn(q, p[k], A.gwb[k]);
    const float2 inner = __ffma2_rn(bno, p[k], __fmul2_rn(anf, e1[k]));
    const float2 w = __fmul2_rn(__fmul2_rn(q, c[k]), inner);
    A.gd[k][0] = __ffma2_rn(w, gx, A.gd[k][0]);
    A.gd[k][1] = __ffma2_rn(w, gy, A.gd[k][1]);
    A.gd[k][2] = __ffma2_rn(w, gz, A.gd[k][2]);
  }
}

// Packed steps over n pairs of b = 0 measurements: every compartment signal of Eqs. 4-5 is
// exactly 1 there (c no longer matters), so y_hat = S0 * sum of the fractions, and each
// accumulator sum_n r E gains sum_n r while the direction terms gain nothing. The sum of the
// fractions is formed again at each pair (a loop-carried copy costs registers the main loop
// needs).
template <int K>
__device__ __forceinline__ void step2_b0(const VoxP<K>& D, const float2* __restrict__ yc2, int stride, int n,
                                         AccP<K>& A) {
  float2 rs = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    float2 T = __fadd2_rn(D.fcsf, D.fgm);
    T = __fadd2_rn(T, D.fres);
#pragma unroll
    for (int k = 0; k < K; ++k) T = __fadd2_rn(T, __fadd2_rn(D.ffin[k], D.fomf[k]));
    const float2 r = __ffma2_rn(D.nS0, T, yc2[i * stride]);   // y - y_hat
    A.l1 = __ffma2_rn(r, r, A.l1);
    rs = __fadd2_rn(rs, r);
  }
  A.gcsf = __fadd2_rn(A.gcsf, rs);
  A.ggm = __fadd2_rn(A.ggm, rs);
  A.gres = __fadd2_rn(A.gres, rs);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    A.gwa[k] = __fadd2_rn(A.gwa[k], rs);
    A.gwb[k] = __fadd2_rn(A.gwb[k], rs);
  }
}

// Fold packed accumulators into the scalar ones (dJ/dS0 from the compartment sums:
// sum_n q T = f_csf sum q E_csf + ... + sum_k (f_k f_in sum q e1 + f_k (1-f_in) sum q p)).
template <int K, int LOSS, bool CAL>
__device__ __forceinline__ void accp_fold(const Vox<K>& P, const AccP<K>& B, Acc<K>& A) {
  A.gcsf = -(B.gcsf.x + B.gcsf.y);
  A.ggm = -(B.ggm.x + B.ggm.y);
  A.gres = -(B.gres.x + B.gres.y);
  A.l1 = B.l1.x + B.l1.y;
  if constexpr (LOSS == kLossNLL) {
    A.l2 = B.l2;
    A.l3 = B.l3;
  }
  if constexpr (CAL) A.u = -(B.u.x + B.u.y);
  float g = P.f[0] * A.gcsf + P.f[1] * A.ggm + P.f[K + 2] * A.gres;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    A.gwa[k] = -(B.gwa[k].x + B.gwa[k].y);
    A.gwb[k] = -(B.gwb[k].x + B.gwb[k].y);
#pragma unroll
    for (int c = 0; c < 3; ++c) A.gd[k][c] = -(B.gd[k][c].x + B.gd[k][c].y);
    g = fmaf(P.f[2 + k] * P.fin, A.gwa[k], fmaf(P.f[2 + k] * P.omf, A.gwb[k], g));
  }
  A.gS0 = g;
}

// The packed accumulators' sums (accp_fold without the S0 term, which needs the voxel's
// transform): for several lanes per voxel, whose sums are combined before the transform.
template <int K, int LOSS, bool CAL>
__device__ __forceinline__ void accp_sums(const AccP<K>& B, Acc<K>& A) {
  A.gS0 = 0.f;
  A.gcsf = -(B.gcsf.x + B.gcsf.y);
  A.ggm = -(B.ggm.x + B.ggm.y);
  A.gres = -(B.gres.x + B.gres.y);
  A.l1 = B.l1.x + B.l1.y;
  if constexpr (LOSS == kLossNLL) {
    A.l2 = B.l2;
    A.l3 = B.l3;
  }
  if constexpr (CAL) A.u = -(B.u.x + B.u.y);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    A.gwa[k] = -(B.gwa[k].x + B.gwa[k].y);
    A.gwb[k] = -(B.gwb[k].x + B.gwb[k].y);
#pragma unroll
    for (int c = 0; c < 3; ++c) A.gd[k][c] = -(B.gd[k][c].x + B.gd[k][c].y);
  }
}

// sum_n q_n T_n from the per-compartment sums (T = sum of fraction-weighted compartment signals).
template <int K>
__device__ __forceinline__ float acc_gS0(const Vox<K>& P, const Acc<K>& A) {
  float g = P.f[0] * A.gcsf + P.f[1] * A.ggm + P.f[K + 2] * A.gres;
#pragma unroll
  for (int k = 0; k < K; ++k) g = fmaf(P.f[2 + k] * P.fin, A.gwa[k], fmaf(P.f[2 + k] * P.omf, A.gwb[k], g));
  return g;
}

// Accumulators of a tile's voxels in shared memory, field-major: s[f * TV + v], 8 + 5K fields.
template <int K>
__device__ __forceinline__ void acc_put(const Acc<K>& A, float* s, int TV, int v) {
  s[0 * TV + v] = A.gS0;
  s[1 * TV + v] = A.gcsf;
  s[2 * TV + v] = A.ggm;
  s[3 * TV + v] = A.gres;
  s[4 * TV + v] = A.l1;
  s[5 * TV + v] = A.l2;
  s[6 * TV + v] = A.l3;
  s[7 * TV + v] = A.u;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    s[(8 + 5 * k) * TV + v] = A.gwa[k];
    s[(9 + 5 * k) * TV + v] = A.gwb[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) s[(10 + 5 * k + c) * TV + v] = A.gd[k][c];
  }
}

template <int K>
__device__ __forceinline__ void acc_get(Acc<K>& A, const float* s, int TV, int v) {
  A.gS0 = s[0 * TV + v];
  A.gcsf = s[1 * TV + v];
  A.ggm = s[2 * TV + v];
  A.gres = s[3 * TV + v];
  A.l1 = s[4 * TV + v];
  A.l2 = s[5 * TV + v];
  A.l3 = s[6 * TV + v];
  A.u = s[7 * TV + v];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    A.gwa[k] = s[(8 + 5 * k) * TV + v];
    A.gwb[k] = s[(9 + 5 * k) * TV + v];
#pragma unroll
    for (int c = 0; c < 3; ++c) A.gd[k][c] = s[(10 + 5 * k + c) * TV + v];
  }
}

// Scaled data-term gradient w.r.t. transformed parameters.
template <int K>
__device__ __forceinline__ void data_grad(const Vox<K>& P, const Acc<K>& A, float scale, float& gS0,
                                          float (&gf)[K + 3], float (&gd)[K][3], float& gfin) {
  const float sS = scale * P.S0;
  gS0 = A.gS0 * scale;
  gf[0] = A.gcsf * sS;
  gf[1] = A.ggm * sS;
  gf[K + 2] = A.gres * sS;
  float gin = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    gf[2 + k] = fmaf(P.fin, A.gwa[k], P.omf * A.gwb[k]) * sS;   // sum q E_wm,k
    gin = fmaf(P.f[2 + k], A.gwa[k] - A.gwb[k], gin);          // sum q sum_k f_k (e1 - p)
    const float w = sS * P.f[2 + k];
#pragma unroll
    for (int c = 0; c < 3; ++c) gd[k][c] = A.gd[k][c] * w;
  }
  gfin = gin * sS;
}

__device__ __forceinline__ void block_reduce3(double v0, double v1, double v2, double (*s_red)[3],
                                              double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v0 = warp_sum_d(v0);
  v1 = warp_sum_d(v1);
  v2 = warp_sum_d(v2);
  if (lane == 0) {
    s_red[warp][0] = v0;
    s_red[warp][1] = v1;
    s_red[warp][2] = v2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0, c = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
      a += s_red[w][0];
      b += s_red[w][1];
      c += s_red[w][2];
    }
    out[0] = a;
    out[1] = b;
    out[2] = c;
  }
}

// ---------------------------------------------------------------------------
// Shell loop (one thread per voxel, MSE, no calibration): the group's measurements are in
// b-value order, so runs of equal b (shells, ShellRun) share Eq. 4's isotropic decays and Eq.
// 5's exponent constants. Per shell and voxel the isotropic mixture T0 is formed once and the
// isotropic adjoint sums need only sum_n r over the shell; per measurement and fiber the two
// exponentials come from the scaled cosine c' = g' . d of the table's g' = s g (see ShellRun):
//   m = c'^2 - log2 f_in,  f_in e1 = 2^(-m),  (1 - f_in) p = 2^(-rho m + Kp),
//   r = y - S0 T = (y - S0 T0) - sum_k S0 f_k (f_in e1 + (1 - f_in) p)  (two measurements per step).
// The adjoint sums are ga_k = sum r f_in e1, gb_k = sum r (1 - f_in) p and
// gd_k = sum r c' (f_in e1 + rho (1 - f_in) p) g', which is -1 / (2 ln 2) times sum r dE_wm,k/dd.
// Per-voxel scalars needed only at shell changes sit in a per-thread column of shared memory.
// ---------------------------------------------------------------------------
constexpr int kFusedThreadsShell = 128;   // threads of the fused kernel's CTA (kFusedThreads)

template <int K>
struct ShellState {
  float2 nf[K];         // -S0 f_wm,k (duplicated)
  float2 dp[K][3];      // d_k (duplicated)
  float2 nlfin;         // -log2 f_in
  float2 c0;            // -S0 T0, T0 the shell's isotropic mixture (b = 0: the sum of all fractions)
  float2 Kp;            // C0 - b D_perp log2(e)
  float2 l1, Qs;        // sum r^2; sum r over the current shell
  float2 ga[K], gb[K];
  float2 gd[K][3];
  int ri, pend, b0;     // current shell, its end pair, b = 0 flag
};

// Rows of a thread's shared-memory column (stride kFusedThreads): S0, f_csf, f_gm, f_res, f_in,
// 1 - f_in, C0, then the sums sum_n r E_csf, sum_n r E_gm, sum_n r E_res.
template <int K>
struct ShellRows {
  static constexpr int s0 = 0, fcsf = 1, fgm = 2, fres = 3, fin = 4, omf = 5, c0 = 6, gcsf = 7, ggm = 8, gres = 9,
                       count = kShellCols;
  static_assert(gres < count, "the column holds every row");
};

template <int K>
__device__ __forceinline__ void shell_step(ShellState<K>& S, float2 gx, float2 gy, float2 gz, float2 y) {
  const float2 nrho = make_float2(-kRho, -kRho), rho = make_float2(kRho, kRho);
  float2 cp[K], e1[K], pp[K], t[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    cp[k] = __ffma2_rn(S.dp[k][0], gx, __ffma2_rn(S.dp[k][1], gy, __fmul2_rn(S.dp[k][2], gz)));
    const float2 m = __ffma2_rn(cp[k], cp[k], S.nlfin);
    e1[k] = make_float2(ex2f_(-m.x), ex2f_(-m.y));
    pp[k] = ex2_2(__ffma2_rn(nrho, m, S.Kp));
    t[k] = __fadd2_rn(e1[k], pp[k]);
  }
  float2 r = __fadd2_rn(y, S.c0);   // y - y_hat
#pragma unroll
  for (int k = 0; k < K; ++k) r = __ffma2_rn(S.nf[k], t[k], r);
  S.l1 = __ffma2_rn(r, r, S.l1);
  S.Qs = __fadd2_rn(S.Qs, r);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    S.ga[k] = __ffma2_rn(r, e1[k], S.ga[k]);
    S.gb[k] = __ffma2_rn(r, pp[k], S.gb[k]);
    const float2 inner = __ffma2_rn(rho, pp[k], e1[k]);
    const float2 w = __fmul2_rn(__fmul2_rn(r, cp[k]), inner);
    S.gd[k][0] = __ffma2_rn(w, gx, S.gd[k][0]);
    S.gd[k][1] = __ffma2_rn(w, gy, S.gd[k][1]);
    S.gd[k][2] = __ffma2_rn(w, gz, S.gd[k][2]);
  }
}

// Closes the current shell: its sum_n r goes into the isotropic sums (and, at b = 0, where
// f_in e1 = f_in and (1 - f_in) p = 1 - f_in, into ga / gb).
template <int K>
__device__ __forceinline__ void shell_close(ShellState<K>& S, const ShellRun& R, float* col) {
  using SR = ShellRows<K>;
  const float q = S.Qs.x + S.Qs.y;
  col[SR::gcsf * kFusedThreadsShell] = fmaf(R.ecsf, q, col[SR::gcsf * kFusedThreadsShell]);
  col[SR::ggm * kFusedThreadsShell] = fmaf(R.egm, q, col[SR::ggm * kFusedThreadsShell]);
  col[SR::gres * kFusedThreadsShell] = fmaf(R.eres, q, col[SR::gres * kFusedThreadsShell]);
  if (R.b0) {
    const float2 fi = dup2(col[SR::fin * kFusedThreadsShell]), om = dup2(col[SR::omf * kFusedThreadsShell]);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      S.ga[k] = __ffma2_rn(fi, S.Qs, S.ga[k]);
      S.gb[k] = __ffma2_rn(om, S.Qs, S.gb[k]);
    }
  }
  S.Qs = make_float2(0.f, 0.f);
}

// Opens shell R: the residual's constant -S0 T0 (T0 the shell's isotropic mixture, at b = 0 the
// sum of every fraction) and the exponent offset Kp.
template <int K>
__device__ __forceinline__ void shell_open(ShellState<K>& S, const ShellRun& R, const float* col) {
  using SR = ShellRows<K>;
  constexpr int C = kFusedThreadsShell;
  S.pend = R.p1;
  S.b0 = R.b0;
  const float T0 = fmaf(col[SR::fcsf * C], R.ecsf, fmaf(col[SR::fgm * C], R.egm, col[SR::fres * C] * R.eres));
  float c0 = -col[SR::s0 * C] * T0;
  if (R.b0) {
#pragma unroll
    for (int k = 0; k < K; ++k) c0 += S.nf[k].x;
  }
  S.c0 = dup2(c0);
  S.Kp = dup2(col[SR::c0 * C] + R.nbperp);
}

// Voxel set-up of the shell loop from the transformed parameters (its column and registers).
template <int K>
__device__ __forceinline__ void shell_begin(ShellState<K>& S, const Vox<K>& P, float* col) {
  using SR = ShellRows<K>;
  constexpr int C = kFusedThreadsShell;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    S.nf[k] = dup2(-P.S0 * P.f[2 + k]);
#pragma unroll
    for (int c = 0; c < 3; ++c) S.dp[k][c] = dup2(P.d[k][c]);
  }
  // log2 f_in and log2(1 - f_in), floored so that a saturated f_in gives no inf - inf
  const float lfin = fmaxf(lg2f_(P.fin), -40.f), lomf = fmaxf(lg2f_(P.omf), -126.f);
  S.nlfin = dup2(-lfin);
  col[SR::s0 * C] = P.S0;
  col[SR::fcsf * C] = P.f[0];
  col[SR::fgm * C] = P.f[1];
  col[SR::fres * C] = P.f[K + 2];
  col[SR::fin * C] = P.fin;
  col[SR::omf * C] = P.omf;
  col[SR::c0 * C] = fmaf(-kRho, lfin, lomf);
  col[SR::gcsf * C] = col[SR::ggm * C] = col[SR::gres * C] = 0.f;
  const float2 z = make_float2(0.f, 0.f);
  S.l1 = S.Qs = z;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    S.ga[k] = S.gb[k] = z;
    S.gd[k][0] = S.gd[k][1] = S.gd[k][2] = z;
  }
  S.ri = -1;
  S.pend = 0;
  S.b0 = 0;
}

// The shell loop's sums as the (unscaled, q = y_hat - y) accumulators of the epilogue:
// gwa_k = sum q f_in e1, gwb_k = sum q (1 - f_in) p (the scaled forms), gS0 = sum q T.
template <int K>
__device__ __forceinline__ void shell_fold(const Vox<K>& P, const ShellState<K>& S, const float* col, Acc<K>& A) {
  using SR = ShellRows<K>;
  constexpr int C = kFusedThreadsShell;
  A.gcsf = -col[SR::gcsf * C];
  A.ggm = -col[SR::ggm * C];
  A.gres = -col[SR::gres * C];
  A.l1 = S.l1.x + S.l1.y;
  float g = P.f[0] * A.gcsf + P.f[1] * A.ggm + P.f[K + 2] * A.gres;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    A.gwa[k] = -(S.ga[k].x + S.ga[k].y);
    A.gwb[k] = -(S.gb[k].x + S.gb[k].y);
#pragma unroll
    for (int c = 0; c < 3; ++c) A.gd[k][c] = kTwoLn2 * (S.gd[k][c].x + S.gd[k][c].y);
    g = fmaf(P.f[2 + k], A.gwa[k] + A.gwb[k], g);
  }
  A.gS0 = g;
}

// Scaled data-term gradient from the shell loop's sums; gu is w.r.t. the raw u of f_in:
// dE_wm/du = f_in (1 - f_in) (e1 - p) = (1 - f_in) (f_in e1) - f_in ((1 - f_in) p).
template <int K>
__device__ __forceinline__ void data_grad_shell(const Vox<K>& P, const Acc<K>& A, float scale, float& gS0,
                                                float (&gf)[K + 3], float (&gd)[K][3], float& gu) {
  const float sS = scale * P.S0;
  gS0 = A.gS0 * scale;
  gf[0] = A.gcsf * sS;
  gf[1] = A.ggm * sS;
  gf[K + 2] = A.gres * sS;
  float gin = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    gf[2 + k] = (A.gwa[k] + A.gwb[k]) * sS;
    gin = fmaf(P.f[2 + k], fmaf(P.omf, A.gwa[k], -P.fin * A.gwb[k]), gin);
    const float w = sS * P.f[2 + k];
#pragma unroll
    for (int c = 0; c < 3; ++c) gd[k][c] = A.gd[k][c] * w;
  }
  gu = gin * sS;
}

// ===========================================================================
// Fused iteration: one persistent kernel over the tile queue does synthesis,
// calibration, data term, adjoint, priors, chain rule and the voxel Adam update.
//
// Each warp streams the signal of its own VW voxels (a contiguous [NP][VW] slice of
// the tile's packed block) through a private ring of NS shared-memory buffers of
// kChunk measurements, refilled by its lane 0 with bulk TMA copies (cp.async.bulk)
// tracked by per-stage mbarriers. The stream runs across tile boundaries: while a
// warp finishes a tile it already fetches the first chunks of the CTA's next tile.
// The measurement table and the bias grid arrive by bulk copy when the group changes.
// ===========================================================================
constexpr int kChunk = 32;    // measurements per ring stage
constexpr int kCalG = 4;      // measurements per warp reduce-scatter of the calibration partials
constexpr int kStages = 2;    // ring depth per warp
constexpr int kFusedThreads = 128;
static_assert(kFusedThreads == kFusedThreadsShell, "the shell loop's shared-memory columns use the CTA size");

// Adam / Rprop state of one voxel. Every load is issued before any store of the update (the
// stores could alias the loads as far as the compiler knows, which would serialise one memory
// round trip per parameter).
template <int Q>
__device__ __forceinline__ void load_moments(const IterArgs& a, int slot, bool writer, float (&mq)[Q],
                                             float (&vq)[Q]) {
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const size_t ix = static_cast<size_t>(q) * a.Vpad + slot;
    mq[q] = writer ? a.m[ix] : 0.f;
    vq[q] = writer ? a.v[ix] : 0.f;
  }
}

// Last CTA of an uncalibrated fused iteration: fixed-order sums of the tiles' partials per
// group (strided over threads, then a fixed tree), the objective and its history, Adam on
// sigma_log for the Rician NLL, the step counter and the next iteration's Adam constants.
__device__ __forceinline__ void finalize_groups(const IterArgs& a, double (*s_sum)[kFusedThreads]) {
  const int tid = threadIdx.x;
  const int step = *a.step;
  bool bad = false;
  for (int gi = 0; gi < a.G; ++gi) {
    const GroupDev gr = a.groups[gi];
    double l = 0.0, sg = 0.0, pr = 0.0;
#pragma unroll 8
    for (int t = gr.tile0 + tid; t < gr.tile0 + gr.ntiles; t += kFusedThreads) {
      l += __ldcg(&a.tile_red[4 * static_cast<size_t>(t)]);
      sg += __ldcg(&a.tile_red[4 * static_cast<size_t>(t) + 1]);
      pr += __ldcg(&a.tile_red[4 * static_cast<size_t>(t) + 2]);
    }
    s_sum[0][tid] = l;
    s_sum[1][tid] = sg;
    s_sum[2][tid] = pr;
    __syncthreads();
    for (int o = kFusedThreads / 2; o > 0; o >>= 1) {
      if (tid < o) {
        s_sum[0][tid] += s_sum[0][tid + o];
        s_sum[1][tid] += s_sum[1][tid + o];
        s_sum[2][tid] += s_sum[2][tid + o];
      }
      __syncthreads();
    }
    if (tid == 0) {
      const double J = s_sum[0][0] + s_sum[2][0];
      a.gloss[gi] = J;
      a.hist[static_cast<size_t>(step % a.hist_len) * a.G + gi] = J;
      if (!isfinite(J)) bad = true;
      if (a.loss_mode == kLossNLL) {
        const int i = gr.gp_off;
        const float gsig = static_cast<float>(s_sum[1][0]);
        if (a.optimizer == 0) {
          const float mq = fmaf(a.beta1, a.gm[i], (1.f - a.beta1) * gsig);
          const float vq = fmaf(a.beta2, a.gv[i], (1.f - a.beta2) * gsig * gsig);
          a.gm[i] = mq;
          a.gv[i] = vq;
          a.gparams_rw[i] -= a.adamc[0] * mq / fmaf(sqrtf(vq), a.adamc[1], a.eps);
        } else {
          float th = a.gparams_rw[i], mq = a.gm[i], vq = a.gv[i];
          rprop_update(th, mq, vq, gsig, a.lr, a.eta_minus, a.eta_plus, a.step_min, a.step_max);
          a.gparams_rw[i] = th;
          a.gm[i] = mq;
          a.gv[i] = vq;
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (bad) atomicOr(a.status, kStNonfinite);
    *const_cast<int32_t*>(a.step) = step + 1;
    const double t2 = static_cast<double>(step) + 2.0;
    float* ac = const_cast<float*>(a.adamc);
    ac[0] = static_cast<float>(a.lr / (1.0 - pow(static_cast<double>(a.beta1), t2)));
    ac[1] = static_cast<float>(1.0 / sqrt(1.0 - pow(static_cast<double>(a.beta2), t2)));
  }
}

// Whether the fused kernel takes two measurements per step in f32x2 arithmetic: with one or
// four lanes per voxel, except the calibrated NLL with five fibers (its packed form spills even
// at 170 registers and measured 11 % slower). Sixteen lanes per voxel (one pair per lane and
// chunk): never, the scalar loop measured 0-20 % faster.
template <int K, int TPV, int LOSS, bool CAL>
__host__ __device__ constexpr bool fused_packed() {
  return (TPV == 1 || TPV == 4) && !(CAL && LOSS == kLossNLL && K >= 5);
}

// CTAs per SM the fused kernel is compiled for: 4 (128 registers per thread) where the voxel
// state fits, 3 (170 registers) for five fibers and the packed NLL and calibrated variants,
// which spill at 128 and measured 7-54 % faster at 3.
template <int K, int TPV, int LOSS, bool CAL>
constexpr int fused_min_blocks() {
  return ((K >= 5) || (fused_packed<K, TPV, LOSS, CAL>() && (CAL || LOSS == kLossNLL))) ? 3 : 4;
}

// SHELL: the shell loop (see ShellState) instead of the packed pairs; only for one thread per
// voxel, the MSE, no calibration and K <= 3, with every group's shells of even length.
template <int K, int TPV, int LOSS, bool CAL, bool SHELL = false>
__global__ void __launch_bounds__(kFusedThreads, (fused_min_blocks<K, TPV, LOSS, CAL>())) k_iter_fused(const IterArgs a) {
  constexpr int NF = K + 3, Q = 4 * K + 5, XF = 4 * K + 3;
  constexpr int NW = kFusedThreads / 32;
  constexpr int VW = 32 / TPV;              // voxels per warp
  constexpr bool PACKED = fused_packed<K, TPV, LOSS, CAL>();
  constexpr bool HOIST = PACKED && TPV == 1 && K <= 3 && LOSS == kLossMSE && !CAL;
  static_assert(!SHELL || HOIST, "the shell loop covers one thread per voxel, MSE, no calibration, K <= 3");
  using SR = ShellRows<(K <= 3 ? K : 3)>;
  // ring stages per warp (kStages; a ring as deep in bytes for four or sixteen lanes per voxel,
  // kStages * TPV, measured 0-25 % slower)
  constexpr int NS = kStages;
  static_assert(kChunk % TPV == 0, "chunk must split evenly across the voxel's lanes");
  extern __shared__ __align__(16) unsigned char smem[];
  const int Vp = a.Vpad;
  MeasRow* s_tab = reinterpret_cast<MeasRow*>(smem);
  // shell loop: [3][Nmax] gradient rows, kMaxRuns shells, the threads' columns, then the ring
  float* s_g = reinterpret_cast<float*>(smem);
  ShellRun* s_runs = reinterpret_cast<ShellRun*>(s_g + 3 * a.Nmax);
  float* s_col = reinterpret_cast<float*>(s_runs + kMaxRuns);
  float* s_ring = SHELL ? s_col + SR::count * kFusedThreads
                        : reinterpret_cast<float*>(s_tab + a.Nmax);       // [NW][NS][kChunk][VW]
  float* s_blr = s_ring + NW * NS * kChunk * VW;                       // [512] (calibration)
  float* s_ab = s_blr + (CAL ? kNGrid : 0);                                 // [NW][2][Nmax] (calibration)
  __shared__ uint64_t s_bar;                 // table / bias grid
  __shared__ uint64_t s_full[NW][NS];
  __shared__ int s_first, s_next;
  __shared__ double s_red[8][3];
  // several lanes per voxel: the tile's reduced accumulators, handed to the epilogue threads
  constexpr int TV = kFusedThreads / TPV;
  __shared__ float s_acc[(TPV > 1) ? (8 + 5 * K) * TV : 1];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // A voxel's TPV lanes lie VW apart (lane = js * VW + lv): the lanes that read one table row
  // at a time are then contiguous, so table reads stay broadcasts and signal reads contiguous.
  const int lv = (TPV == 1) ? lane : lane % VW, js = (TPV == 1) ? 0 : lane / VW;
  const int vl = (TPV == 1) ? tid : warp * VW + lv;
  const int step = *a.step;
  const int par = step & 1;
  const float* xf_cur = a.xf + static_cast<size_t>(par) * XF * Vp;
  float* xf_nxt = a.xf + static_cast<size_t>(par ^ 1) * XF * Vp;
  float* ring = s_ring + warp * (NS * kChunk * VW);
  if (tid == 0) {
    mbar_init(&s_bar, 1);
    for (int w = 0; w < NW; ++w)
      for (int s = 0; s < NS; ++s) mbar_init(&s_full[w][s], 1);
    fence_mbar_init();
    const int q = atomicAdd(a.queue, 1);
    s_first = (q < a.ntiles) ? a.tile_order[q] : a.ntiles;
  }
  __syncthreads();
  const float stepsz = a.adamc[0], isbc2 = a.adamc[1];
  int cur_group = -1;
  uint32_t tphase = 0;
  uint32_t g = 0;      // stream chunks consumed by this warp
  uint32_t iss = 0;    // stream chunks issued by this warp (lane 0's copy is authoritative)
  uint32_t base = 0;   // stream position of the current tile's chunk 0
  bool failed = false;
  int t = s_first;
  // launched as a programmatic dependent of k_prior_grad, this grid can start while that one
  // finishes: its rows are read only in the epilogue, so each thread waits once, before its
  // first epilogue (no write before that point is read by k_prior_grad)
  bool dep_done = false;

  // Lane 0: issue stream position `pos` = chunk j of the tile at y_off (NP padded rows).
  auto issue = [&](uint32_t pos, int64_t y_off, int NP, int j) {
    const int s = pos % NS;
    const int cnt = min(kChunk, NP - j * kChunk);
    const uint32_t bytes = static_cast<uint32_t>(cnt) * VW * 4u;
    const float* src = a.y + y_off + static_cast<int64_t>(warp) * NP * VW + static_cast<int64_t>(j) * kChunk * VW;
    fence_proxy_async_smem();
    mbar_expect_tx(&s_full[warp][s], bytes);
    tma_bulk_g2s(ring + s * (kChunk * VW), src, bytes, &s_full[warp][s]);
  };

  while (t < a.ntiles) {
    if (tid == 0) {
      const int q = atomicAdd(a.queue, 1);
      s_next = (q < a.ntiles) ? a.tile_order[q] : a.ntiles;
    }
    __syncthreads();
    const int t_next = s_next;
    const Tile tl = a.tiles[t];
    const GroupDev gr = a.groups[tl.group];
    const int N = tl.n_meas, NP = (N + 3) & ~3;
    const int nch = (NP + kChunk - 1) / kChunk;
    int64_t ny_off = 0;
    int nNP = 0, nnch = 0;
    if (t_next < a.ntiles) {
      const Tile tn = a.tiles[t_next];
      ny_off = tn.y_off;
      nNP = (tn.n_meas + 3) & ~3;
      nnch = (nNP + kChunk - 1) / kChunk;
    }
    if (tl.group != cur_group) {
      if (tid == 0) {
        fence_proxy_async_smem();
        if (SHELL) {
          const uint32_t gb = 3u * static_cast<uint32_t>(NP) * 4u;
          const uint32_t rb = static_cast<uint32_t>(gr.n_runs) * static_cast<uint32_t>(sizeof(ShellRun));
          mbar_expect_tx(&s_bar, gb + rb);
          tma_bulk_g2s(s_g, a.gtab + gr.gtab_off, gb, &s_bar);
          tma_bulk_g2s(s_runs, a.runs + gr.run_off, rb, &s_bar);
        } else if (PACKED) {
          const uint32_t tb = static_cast<uint32_t>(NP / 2 * sizeof(MeasPair));
          mbar_expect_tx(&s_bar, tb + (CAL ? kNGrid * 4u : 0u));
          tma_bulk_g2s(s_tab, a.table2 + gr.table2_off, tb, &s_bar);
          if (CAL) tma_bulk_g2s(s_blr, a.gparams + gr.gp_off + 4 + 2 * gr.N4, kNGrid * 4u, &s_bar);
        } else {
          const uint32_t tb = static_cast<uint32_t>(N * sizeof(MeasRow));
          mbar_expect_tx(&s_bar, tb + (CAL ? kNGrid * 4u : 0u));
          tma_bulk_g2s(s_tab, a.table + gr.table_off, tb, &s_bar);
          if (CAL) tma_bulk_g2s(s_blr, a.gparams + gr.gp_off + 4 + 2 * gr.N4, kNGrid * 4u, &s_bar);
        }
      }
      if (!failed && !mbar_wait(&s_bar, tphase)) {
        if (tid == 0) atomicOr(a.status, kStTimeout);
        failed = true;
      }
      tphase ^= 1;
      cur_group = tl.group;
    }
    // L2 prefetch of the per-voxel rows a tile reads (parameters, Adam moments, prior data):
    // for the first tile now, and for the next tile one whole tile ahead of its use
    if (tid == 32) {
      const uint32_t rb = static_cast<uint32_t>(kFusedThreads / TPV) * 4u;
      auto rows = [&](int slot0) {
        for (int q = 0; q < Q; ++q) {
          const size_t o = static_cast<size_t>(q) * Vp + slot0;
          prefetch_l2(a.theta + o, rb);
          prefetch_l2(a.m + o, rb);
          prefetch_l2(a.v + o, rb);
        }
        if (a.nb_priors) {
          for (int c = 0; c < kPgRows<K>; ++c) prefetch_l2(a.pg + static_cast<size_t>(c) * Vp + slot0, rb);
        } else if (a.nb_priors) {
          for (int e = 0; e < a.n_nbr; ++e) prefetch_l2(a.nbr + static_cast<size_t>(e) * Vp + slot0, rb);
          if (a.lam_sp > 0.f)
            for (int c = 0; c < NF; ++c) prefetch_l2(a.hsp + static_cast<size_t>(c) * Vp + slot0, rb);
        }
      };
      if (t == s_first) rows(tl.slot0);
      if (t_next < a.ntiles) rows(t_next * (kFusedThreads / TPV));
    }

    const int slot = tl.slot0 + vl;
    const bool act = vl < tl.count;
    Vox<K> P;
    {
      float th[Q];
      load_theta<K>(a.theta, Vp, slot, act, th);
      transform<K>(th, P);
    }
    float inv_s2 = 0.f, slog = 0.f;
    if (LOSS == kLossNLL) {
      slog = a.gparams[gr.gp_off];
      inv_s2 = expf(-2.f * slog);
    }
    const float scale = (LOSS == kLossMSE) ? 2.f * gr.inv_M : inv_s2;
    float B = 1.f;
    int cx = 0, cy = 0, cz = 0;
    if (CAL) {
      unpack_coord(act ? a.vcoord[slot] : 0u, cx, cy, cz);
      B = expf(tri_eval(s_blr, tri_weights(cx, cy, cz, gr.nx, gr.ny, gr.nz)));
    }
    Acc<K> A;
    acc_zero<K>(A);
    float ffin[K], fomf[K];
    fiber_weights<K>(P, ffin, fomf);
    VoxP<K> DP;
    AccP<K> AP;
    ShellState<(K <= 3 ? K : 3)> SS;
    float* col = s_col + tid;
    if constexpr (SHELL) {
      shell_begin(SS, P, col);
    } else if constexpr (PACKED) {
      voxp_init<K>(P, DP, AP);
    }
    for (int j = 0; j < nch; ++j) {
      if (lane == 0) {
        // keep NS chunks of this warp's stream in flight (this tile, then the next)
        while (iss < g + NS) {
          const uint32_t r = iss - base;
          if (r < static_cast<uint32_t>(nch)) issue(iss, tl.y_off, NP, r);
          else if (r - nch < static_cast<uint32_t>(nnch)) issue(iss, ny_off, nNP, r - nch);
          else break;
          ++iss;
        }
      }
      const int s = g % NS;
      if (!failed && !mbar_wait(&s_full[warp][s], (g / NS) & 1)) {
        atomicOr(a.status, kStTimeout);
        failed = true;
      }
      const int cnt = min(kChunk, N - j * kChunk);
      if constexpr (SHELL) {
        // pairs of this chunk, in segments that stay inside one shell (shells have even lengths)
        const float2* __restrict__ yc2 = reinterpret_cast<const float2*>(ring + s * (kChunk * VW)) + lv;
        // gradient rows: {g_x, g_y} of a pair as one float4, then the g_z pairs
        const float4* __restrict__ gxy = reinterpret_cast<const float4*>(s_g);
        const float2* __restrict__ gz2 = reinterpret_cast<const float2*>(s_g + 2 * NP);
        const int pc0 = j * (kChunk / 2), pc1 = min(pc0 + kChunk / 2, N / 2);
        if (act) {
          int p = pc0;
          while (p < pc1) {
            if (p >= SS.pend) {
              // every pass either opens a shell (at most n_runs) or advances p, so this ends
              // even for a table that did not cover the pairs
              if (SS.ri + 1 >= gr.n_runs) break;
              if (SS.ri >= 0) shell_close(SS, s_runs[SS.ri], col);
              ++SS.ri;
              shell_open(SS, s_runs[SS.ri], col);
              continue;
            }
            const int pe = min(pc1, SS.pend);
            if (SS.b0) {
#pragma unroll 1
              for (; p < pe; ++p) {
                const float2 r = __fadd2_rn(yc2[(p - pc0) * VW], SS.c0);
                SS.l1 = __ffma2_rn(r, r, SS.l1);
                SS.Qs = __fadd2_rn(SS.Qs, r);
              }
            } else {
              // three steps in flight (on the brain workload unroll 2 / 4 / 8 measured 0.1-0.3 %
              // slower, 6 2.5 % slower; no spills in any)
#pragma unroll 3
              for (; p < pe; ++p) {
                const float4 gq = gxy[p];
                shell_step(SS, make_float2(gq.x, gq.y), make_float2(gq.z, gq.w), gz2[p], yc2[(p - pc0) * VW]);
              }
            }
          }
        }
        __syncwarp();
        ++g;
        continue;
      }
      if constexpr (PACKED) {
        const float2* __restrict__ yc2 = reinterpret_cast<const float2*>(ring + s * (kChunk * VW)) + lv;
        const MeasPair* __restrict__ tab2 = reinterpret_cast<const MeasPair*>(s_tab) + j * (kChunk / 2);
        // leading pairs of b = 0 measurements (the group's table starts with them); the NLL
        // still needs the Bessel terms there, so it takes them as ordinary pairs
        const int i0 = (LOSS == kLossMSE) ? max(0, min(kChunk / 2, gr.nb0p - j * (kChunk / 2))) : 0;
        if constexpr (CAL && TPV == 1) {
          // two packed steps (four measurements) per reduce-scatter of the alpha / beta
          // partials; the accumulators hold the negated values, so the stores negate
          const float2 B2 = make_float2(B, B);
#pragma unroll 1
          for (int i = 0; i < kChunk / 2; i += 2) {
            float uu[4], rv[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int pi = i + h;
              float2 u = make_float2(0.f, 0.f), r = make_float2(0.f, 0.f);
              if (act && 2 * pi < cnt)
                step2<K, true, LOSS, true>(DP, tab2[pi], yc2[pi * VW], make_float2(1.f, (2 * pi + 1 < cnt) ? 1.f : 0.f),
                                           AP, inv_s2, B2, &u, &r);
              uu[2 * h] = u.x;
              uu[2 * h + 1] = u.y;
              rv[2 * h] = r.x;
              rv[2 * h + 1] = r.y;
            }
            const float su = warp_scatter_sum<4>(uu);
            const float sr = warp_scatter_sum<4>(rv);
            const int m = lane >> 3;
            if ((lane & 7) == 0 && 2 * i + m < cnt) {
              s_ab[(warp * 2) * a.Nmax + j * kChunk + 2 * i + m] = -su;
              s_ab[(warp * 2 + 1) * a.Nmax + j * kChunk + 2 * i + m] = -sr;
            }
          }
        } else if constexpr (CAL) {
          // several lanes per voxel: lane js takes pairs js, js + TPV, ...; two packed steps
          // (four measurements) per reduce-scatter over the VW lanes that share js (one per
          // voxel of the warp); value q of a lane is half q & 1 of its step q >> 1
          const float2 B2 = make_float2(B, B);
          constexpr int LVW = (VW == 8) ? 3 : (VW == 16) ? 4 : 5;
#pragma unroll 1
          for (int i = 0; i < kChunk / 2 / TPV; i += 2) {
            float uu[4], rv[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int pi = (i + h) * TPV + js;
              float2 u = make_float2(0.f, 0.f), r = make_float2(0.f, 0.f);
              if (act && 2 * pi < cnt)
                step2<K, true, LOSS, true>(DP, tab2[pi], yc2[pi * VW], make_float2(1.f, (2 * pi + 1 < cnt) ? 1.f : 0.f),
                                           AP, inv_s2, B2, &u, &r);
              uu[2 * h] = u.x;
              uu[2 * h + 1] = u.y;
              rv[2 * h] = r.x;
              rv[2 * h + 1] = r.y;
            }
            const float su = warp_scatter_sum<4, VW>(uu);
            const float sr = warp_scatter_sum<4, VW>(rv);
            const int q = lv >> (LVW - 2);
            const int n = 2 * ((i + (q >> 1)) * TPV + js) + (q & 1);
            if ((lv & ((VW >> 2) - 1)) == 0 && n < cnt) {
              s_ab[(warp * 2) * a.Nmax + j * kChunk + n] = -su;
              s_ab[(warp * 2 + 1) * a.Nmax + j * kChunk + n] = -sr;
            }
          }
        } else if (act && cnt == kChunk && i0 == 0) {
          // lane js of the voxel takes pairs js, js + TPV, ...
          // (with five fibers unrolling spills: one step at a time measured 2-6 % faster)
#pragma unroll (K >= 5 ? 1 : 2)
          for (int i = 0; i < kChunk / 2 / TPV; ++i) {
            const int pi = (TPV == 1) ? i : i * TPV + js;
            step2<K, false, LOSS>(DP, tab2[pi], yc2[pi * VW], make_float2(1.f, 1.f), AP, inv_s2);
          }
        } else if (act && TPV == 1) {
          if (i0 > 0) step2_b0<K>(DP, yc2, VW, i0, AP);
#pragma unroll 1
          for (int i = i0; i < (cnt + 1) / 2; ++i)
            step2<K, true, LOSS>(DP, tab2[i], yc2[i * VW], make_float2(1.f, (2 * i + 1 < cnt) ? 1.f : 0.f), AP,
                                 inv_s2);
        } else if (act) {
          if (i0 > js) step2_b0<K>(DP, yc2 + js * VW, TPV * VW, (i0 - js + TPV - 1) / TPV, AP);
          const int first = i0 + ((js - i0) % TPV + TPV) % TPV;   // this lane's first pair >= i0
#pragma unroll 1
          for (int pi = first; pi < (cnt + 1) / 2; pi += TPV)
            step2<K, true, LOSS>(DP, tab2[pi], yc2[pi * VW], make_float2(1.f, (2 * pi + 1 < cnt) ? 1.f : 0.f), AP,
                                 inv_s2);
        }
        __syncwarp();
        ++g;
        continue;
      }
      // pair-interleaved slice: chunk-relative measurement nl of voxel lv
      const float* __restrict__ yc = ring + s * (kChunk * VW) + 2 * lv;
      const MeasRow* __restrict__ tab = s_tab + j * kChunk;
      if (!CAL && act && cnt == kChunk) {
        // full chunk: no predicates
#pragma unroll
        for (int i = 0; i < kChunk / TPV; ++i) {
          const int nl = i * TPV + js;
          float rr, u;
          pair<K, LOSS, CAL, false>(P, ffin, fomf, tab[nl], yc[(nl >> 1) * (2 * VW) + (nl & 1)], B, inv_s2, 0.f, A, rr, u);
        }
      } else if (CAL && TPV == 1) {
        // per-measurement alpha / beta partials summed over the warp's 32 voxels, kCalG
        // measurements at a time by one reduce-scatter (lane L ends with measurement
        // L / (32 / kCalG) of the group; the first lane of each run of 32 / kCalG stores it)
        constexpr int G = kCalG;
        for (int i0 = 0; i0 < kChunk; i0 += G) {
          float uu[G], rv[G];
#pragma unroll
          for (int gq = 0; gq < G; ++gq) {
            const int nl = i0 + gq;
            const bool ok = act && (nl < cnt);
            float rr = 0.f, u = 0.f;
            if (ok) pair<K, LOSS, CAL, false>(P, ffin, fomf, tab[nl], yc[(nl >> 1) * (2 * VW) + (nl & 1)], B, inv_s2, 0.f, A, rr, u);
            uu[gq] = ok ? u : 0.f;
            rv[gq] = ok ? rr : 0.f;
          }
          const float su = warp_scatter_sum<G>(uu);
          const float sr = warp_scatter_sum<G>(rv);
          const int m = lane >> (G == 8 ? 2 : G == 4 ? 3 : 4);
          if ((lane & (32 / G - 1)) == 0 && i0 + m < cnt) {
            s_ab[(warp * 2) * a.Nmax + j * kChunk + i0 + m] = su;
            s_ab[(warp * 2 + 1) * a.Nmax + j * kChunk + i0 + m] = sr;
          }
        }
      } else {
#pragma unroll 4
        for (int i = 0; i < kChunk / TPV; ++i) {
          const int nl = i * TPV + js;
          const bool ok = act && (nl < cnt);
          float rr = 0.f, u = 0.f;
          if (ok) pair<K, LOSS, CAL, false>(P, ffin, fomf, tab[nl], yc[(nl >> 1) * (2 * VW) + (nl & 1)], B, inv_s2, 0.f, A, rr, u);
          if (CAL) {
            // over the warp's voxels: the VW lanes of one js are contiguous
            float su = warp_sum_range<1, VW / 2>(ok ? u : 0.f);
            float sr = warp_sum_range<1, VW / 2>(ok ? rr : 0.f);
            if (lv == 0 && nl < cnt) {
              s_ab[(warp * 2) * a.Nmax + j * kChunk + nl] = su;
              s_ab[(warp * 2 + 1) * a.Nmax + j * kChunk + nl] = sr;
            }
          }
        }
      }
      __syncwarp();
      ++g;
    }
    base += nch;
    if constexpr (SHELL) {
      if (act && SS.ri >= 0) shell_close(SS, s_runs[SS.ri], col);
    }
    if constexpr (TPV > 1) {
      // sum each voxel's lanes and hand the sums to one epilogue thread: voxel v of the tile
      // goes to thread v, so that a warp's epilogue serves 32 voxels, as with one thread per voxel
      if constexpr (PACKED) accp_sums<K, LOSS, CAL>(AP, A);
      acc_reduce_tpv<K, TPV, VW>(A);
      if (js == 0) acc_put<K>(A, s_acc, TV, vl);
      __syncthreads();
    }
    if (!dep_done) {
      grid_dep_wait();
      dep_done = true;
    }
    // the epilogue's voxel: the thread's own with one thread per voxel, else voxel tid of the
    // tile for the first TV threads (the others skip to the tile partials)
    const bool epi = (TPV == 1) || tid < TV;
    const int eslot = (TPV == 1) ? slot : tl.slot0 + min(tid, TV - 1);
    const bool eact = (TPV == 1) ? act : (tid < tl.count);
    const bool writer = eact && (js == 0 || TPV > 1);
    float dloss = 0.f, dsig = 0.f, ploss = 0.f;
    if (epi) {
      // voxel transforms again (not kept live across the loop). Where registers allow (HOIST),
      // the raw parameters and the moments are read here, once, so that their latency overlaps
      // the epilogue's math; otherwise they are re-read before the update.
      float th[Q], mq[Q], vq[Q];
      load_theta<K>(a.theta, Vp, eslot, eact, th);
      if constexpr (HOIST) load_moments<Q>(a, eslot, writer, mq, vq);
      transform<K>(th, P);
      if constexpr (TPV == 1) {
        if constexpr (SHELL) {
          shell_fold(P, SS, col, A);
        } else if constexpr (PACKED) {
          accp_fold<K, LOSS, CAL>(P, AP, A);
        }
      } else {
        acc_get<K>(A, s_acc, TV, tid);
        if constexpr (PACKED) A.gS0 = acc_gS0<K>(P, A);
        if constexpr (CAL) {
          unpack_coord(eact ? a.vcoord[eslot] : 0u, cx, cy, cz);
          B = expf(tri_eval(s_blr, tri_weights(cx, cy, cz, gr.nx, gr.ny, gr.nz)));
        }
      }

      // ---- data-term gradient and value
      float gS0, gf[NF], gd[K][3], gfin;
      if constexpr (SHELL) {
        data_grad_shell<K>(P, A, scale, gS0, gf, gd, gfin);   // gfin: w.r.t. the raw u
      } else {
        data_grad<K>(P, A, scale, gS0, gf, gd, gfin);
      }
      if (LOSS == kLossMSE) {
        dloss = A.l1 * gr.inv_M;
      } else {
        dloss = 2.f * slog * N + 0.5f * inv_s2 * A.l1 - A.l3;
        dsig = 2.f * N - inv_s2 * (A.l1 + 2.f * A.l2);
      }
      // ---- priors
      ploss = priors<K, true>(a, P, eslot, gr.inv_M, xf_cur, gS0, gf, gd);
      float gUv = A.u * scale;
      if (CAL && a.w_tv > 0.f) {
        const uint32_t fl = eact ? a.vflag[eslot] : 0u;
        ploss += tv_term(s_blr, cx, cy, cz, gr, fl, B, a.w_tv * gr.inv_M, a.tv_eps, gUv);
      }
      // ---- chain rule and the update
      if constexpr (!HOIST) {
        load_theta<K>(a.theta, Vp, eslot, eact, th);
        load_moments<Q>(a, eslot, writer, mq, vq);
      }
      float gq[Q];
      chain_raw<K, SHELL>(P, gS0, gf, gd, gfin, gq);
      if (a.optimizer == 0) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          mq[q] = fmaf(a.beta1, mq[q], (1.f - a.beta1) * gq[q]);
          vq[q] = fmaf(a.beta2, vq[q], (1.f - a.beta2) * gq[q] * gq[q]);
          th[q] -= stepsz * mq[q] * frcp(fmaf(fsqrt(vq[q]), isbc2, a.eps));
        }
      } else {
#pragma unroll
        for (int q = 0; q < Q; ++q)
          rprop_update(th[q], mq[q], vq[q], gq[q], a.lr, a.eta_minus, a.eta_plus, a.step_min, a.step_max);
      }
      if (writer) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const size_t ix = static_cast<size_t>(q) * Vp + eslot;
          a.m[ix] = mq[q];
          a.v[ix] = vq[q];
          a.theta[ix] = th[q];
        }
      }
      if (a.nb_priors && writer) {
        Vox<K> Pn;
        transform<K>(th, Pn);
        store_xf<K>(xf_nxt, Vp, eslot, Pn);
      }
      if (CAL && writer) a.gU[eslot] = gUv;
    }
    // ---- tile partials (fixed-order reductions)
    block_reduce3(writer ? static_cast<double>(dloss) : 0.0, writer ? static_cast<double>(dsig) : 0.0,
                  writer ? static_cast<double>(ploss) : 0.0, s_red, a.tile_red + 4 * static_cast<size_t>(t));
    if (CAL) {
      for (int e = tid; e < 2 * N; e += kFusedThreads) {
        const int w2 = (e < N) ? 0 : 1;
        const int n = e - w2 * N;
        float sum = 0.f;
        for (int w = 0; w < NW; ++w) sum += s_ab[(w * 2 + w2) * a.Nmax + n];
        a.tile_ab[tl.ab_off + e] = sum * scale;
      }
    }
    if (__syncthreads_or(failed)) break;   // block-uniform exit after a timed-out wait
    t = t_next;
  }
  if (failed && lane == 0) {
    // let copies still in flight land before the CTA's shared memory is released
    for (uint32_t p = g; p < iss; ++p) mbar_wait(&s_full[warp][p % NS], (p / NS) & 1);
  }
  // The last CTA to leave resets the queue for the next iteration (and, without
  // calibration, finalises the groups).
  __shared__ int s_last;
  if (tid == 0) {
    __threadfence();
    s_last = (atomicAdd(a.done, 1) == static_cast<int>(gridDim.x) - 1);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (!CAL && a.fold_groups) {
      __shared__ double s_sum[3][kFusedThreads];
      finalize_groups(a, s_sum);
    }
    if (tid == 0) {
      *a.queue = 0;
      *a.done = 0;
      __threadfence();
    }
  }
}

// ===========================================================================
// Plain (unfused) kernels: one launch per step and per patch (tile range).
// ===========================================================================

// Fractions and unit directions for a tile range (slot-parallel).
template <int K>
__global__ void k_transform(const IterArgs a, int tile_begin, int tile_end) {
  const int XF = 4 * K + 3;
  const int slot = tile_begin * a.TV + blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= tile_end * a.TV) return;
  const Tile tl = a.tiles[slot / a.TV];
  if (slot - tl.slot0 >= tl.count) return;
  float th[4 * K + 5];
  load_theta<K>(a.theta, a.Vpad, slot, true, th);
  Vox<K> P;
  transform<K>(th, P);
  store_xf<K>(a.xf + static_cast<size_t>((*a.step) & 1) * XF * a.Vpad, a.Vpad, slot, P);
}

// Readout (Sec. 3 "Configuration": fiber directions are the peaks): unit directions,
// fractions and peak flags (a fiber's share of the WM fraction >= rel_thresh), mask order.
template <int K>
__global__ void k_fibers(const IterArgs a, const int32_t* __restrict__ slot_of_vox, int64_t V, float rel_thresh,
                         float* __restrict__ dirs, float* __restrict__ fracs, uint8_t* __restrict__ peaks) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= V) return;
  float th[4 * K + 5];
  load_theta<K>(a.theta, a.Vpad, slot_of_vox[v], true, th);
  Vox<K> P;
  transform<K>(th, P);
  float wm = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) wm += P.f[2 + k];
  const float inv_wm = 1.f / fmaxf(wm, 1e-12f);
  if (fracs) {
#pragma unroll
    for (int i = 0; i < K + 3; ++i) fracs[v * (K + 3) + i] = P.f[i];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (dirs) {
#pragma unroll
      for (int c = 0; c < 3; ++c) dirs[(v * K + k) * 3 + c] = P.d[k][c];
    }
    if (peaks) peaks[v * K + k] = (P.f[2 + k] * inv_wm >= rel_thresh) ? 1 : 0;
  }
}

// Slab stitching (Sec. 3 "Configuration": overlapping slabs stitched by weighted averaging;
// the ramp weights and the fiber matching are this library's choice). Output voxel v takes
// the estimate at handle voxel src0[v] and, where two slabs overlap, blends in the one at
// src1[v] with weight w1[v] (src0's weight is 1 - w1). The later slab's fibers are matched to
// the earlier slab's by the permutation maximising sum_k |d0_k . d1_pi(k)| (FP64 dot
// products, first maximum in lexicographic order), each matched direction is flipped into
// the same hemisphere, then S0, fractions, f_intra and the directions are averaged and the
// directions renormalised.
template <int K>
__global__ void k_stitch(const IterArgs a, const int32_t* __restrict__ slot_of_vox, int64_t n_out,
                         const int64_t* __restrict__ src0, const int64_t* __restrict__ src1,
                         const float* __restrict__ w1, float* __restrict__ s0, float* __restrict__ fracs,
                         float* __restrict__ fin, float* __restrict__ dirs) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v >= n_out) return;
  float th[4 * K + 5];
  Vox<K> A;
  load_theta<K>(a.theta, a.Vpad, slot_of_vox[src0[v]], true, th);
  transform<K>(th, A);
  float S = A.S0, fi = A.fin, f[K + 3], d[K][3];
#pragma unroll
  for (int i = 0; i < K + 3; ++i) f[i] = A.f[i];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) d[k][c] = A.d[k][c];
  const int64_t b = src1[v];
  if (b >= 0) {
    Vox<K> B;
    load_theta<K>(a.theta, a.Vpad, slot_of_vox[b], true, th);
    transform<K>(th, B);
    double ad[K][K];
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
      for (int j = 0; j < K; ++j)
        ad[i][j] = fabs(static_cast<double>(A.d[i][0]) * B.d[j][0] + static_cast<double>(A.d[i][1]) * B.d[j][1] +
                        static_cast<double>(A.d[i][2]) * B.d[j][2]);
    // lexicographic permutations of 0..K-1 (next-permutation), first strict maximum kept
    int p[K], bp[K];
#pragma unroll
    for (int k = 0; k < K; ++k) p[k] = bp[k] = k;
    double best = -1.0;
    for (;;) {
      double sum = 0.0;
      for (int k = 0; k < K; ++k) sum += ad[k][p[k]];
      if (sum > best) {
        best = sum;
        for (int k = 0; k < K; ++k) bp[k] = p[k];
      }
      int i = K - 2;
      while (i >= 0 && p[i] > p[i + 1]) --i;
      if (i < 0) break;
      int j = K - 1;
      while (p[j] < p[i]) --j;
      int t = p[i];
      p[i] = p[j];
      p[j] = t;
      for (int l = i + 1, r = K - 1; l < r; ++l, --r) {
        t = p[l];
        p[l] = p[r];
        p[r] = t;
      }
    }
    const float wb = w1[v], wa = 1.f - wb;
    S = wa * A.S0 + wb * B.S0;
    fi = wa * A.fin + wb * B.fin;
    f[0] = wa * A.f[0] + wb * B.f[0];
    f[1] = wa * A.f[1] + wb * B.f[1];
    f[K + 2] = wa * A.f[K + 2] + wb * B.f[K + 2];
    for (int k = 0; k < K; ++k) {
      const int m = bp[k];
      const float dot = A.d[k][0] * B.d[m][0] + A.d[k][1] * B.d[m][1] + A.d[k][2] * B.d[m][2];
      const float sg = (dot >= 0.f) ? wb : -wb;
      f[2 + k] = wa * A.f[2 + k] + wb * B.f[2 + m];
      float n2 = 0.f;
      for (int c = 0; c < 3; ++c) {
        d[k][c] = wa * A.d[k][c] + sg * B.d[m][c];
        n2 += d[k][c] * d[k][c];
      }
      const float inv = rsqrtf(fmaxf(n2, kNormEps2));
      for (int c = 0; c < 3; ++c) d[k][c] *= inv;
    }
  }
  if (s0) s0[v] = S;
  if (fin) fin[v] = fi;
  if (fracs) {
#pragma unroll
    for (int i = 0; i < K + 3; ++i) fracs[v * (K + 3) + i] = f[i];
  }
  if (dirs) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) dirs[(v * K + k) * 3 + c] = d[k][c];
  }
}

// Synthesis + calibration: y_hat for every (voxel, measurement) of the tile range.
template <int K, int TPV, bool CAL>
__global__ void __launch_bounds__(256) k_synth(const IterArgs a, const PlainArgs pa) {
  const int t = pa.tile_begin + blockIdx.x;
  if (t >= pa.tile_end) return;
  const Tile tl = a.tiles[t];
  const GroupDev gr = a.groups[tl.group];
  const MeasRow* tab = a.table + gr.table_off;
  const int vl = threadIdx.x / TPV, js = threadIdx.x % TPV;
  if (vl >= tl.count) return;
  const int slot = tl.slot0 + vl;
  float th[4 * K + 5];
  load_theta<K>(a.theta, a.Vpad, slot, true, th);
  Vox<K> P;
  transform<K>(th, P);
  float B = 1.f;
  if (CAL) {
    int x, y, z;
    unpack_coord(a.vcoord[slot], x, y, z);
    B = expf(tri_eval(a.gparams + gr.gp_off + 4 + 2 * gr.N4, tri_weights(x, y, z, gr.nx, gr.ny, gr.nz)));
  }
  for (int n = js; n < tl.n_meas; n += TPV) {
    const MeasRow R = tab[n];
    float T = P.f[0] * R.ecsf;
    T = fmaf(P.f[1], R.egm, T);
    T = fmaf(P.f[K + 2], R.eres, T);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float c = fmaf(P.d[k][0], R.gx, fmaf(P.d[k][1], R.gy, P.d[k][2] * R.gz));
      const float c2 = c * c;
      const float e1 = ex2f_(R.nkpar * c2);
      const float p = ex2f_(fmaf(R.nkd, c2, R.nkperp));
      T = fmaf(P.f[2 + k], fmaf(P.fin, e1, P.omf * p), T);
    }
    const float S = P.S0 * T;
    pa.yhat[ypos(tl, n, vl, a.VW)] = CAL ? fmaf(R.A * B, S, R.beta) : S;
  }
}

// Data term: per-element derivative dL/dy_hat (scaled) and per-tile loss / sigma partials.
template <int LOSS>
__global__ void __launch_bounds__(256) k_loss(const IterArgs a, const PlainArgs pa) {
  __shared__ double s_red[8][3];
  const int t = pa.tile_begin + blockIdx.x;
  if (t >= pa.tile_end) return;
  const Tile tl = a.tiles[t];
  const GroupDev gr = a.groups[tl.group];
  const int N = tl.n_meas;
  float inv_s2 = 0.f, slog = 0.f;
  if (LOSS == kLossNLL) {
    slog = a.gparams[gr.gp_off];
    inv_s2 = expf(-2.f * slog);
  }
  const float scale = (LOSS == kLossMSE) ? 2.f * gr.inv_M : inv_s2;
  double l = 0.0, sg = 0.0;
  for (int e = threadIdx.x; e < N * a.TV; e += blockDim.x) {
    const int n = e / a.TV, vl = e - n * a.TV;
    if (vl >= tl.count) continue;
    const size_t ix = ypos(tl, n, vl, a.VW);
    const float yh = pa.yhat[ix], yv = a.y[ix];
    float rr;
    if (LOSS == kLossMSE) {
      rr = yh - yv;
      l += static_cast<double>(rr * rr) * gr.inv_M;
    } else {
      const float ay = fabsf(yh);
      const float sy = (yh >= 0.f) ? yv : -yv;
      float Qz, Lz;
      bessel_QL<true>(yv * ay * inv_s2, Qz, Lz);
      const float d = yv - ay;
      l += static_cast<double>(2.f * slog + 0.5f * inv_s2 * d * d - Lz);
      sg += static_cast<double>(2.f - inv_s2 * (d * d + 2.f * yv * ay * Qz));
      rr = fmaf(sy, Qz, yh - sy);
    }
    pa.r[ix] = rr * scale;
  }
  double out[3];
  block_reduce3(l, sg, 0.0, s_red, out);
  if (threadIdx.x == 0) {
    a.tile_red[4 * static_cast<size_t>(t) + 0] = out[0];
    a.tile_red[4 * static_cast<size_t>(t) + 1] = out[1];
  }
}

// Adjoint: recomputes the compartment exponentials and back-substitutes the stored
// dL/dy_hat into raw-parameter gradients, alpha/beta partials and dJ/dU.
template <int K, int TPV, bool CAL>
__global__ void __launch_bounds__(256) k_adjoint(const IterArgs a, const PlainArgs pa) {
  constexpr int NF = K + 3, Q = 4 * K + 5;
  extern __shared__ __align__(16) unsigned char smem[];
  float* s_ab = reinterpret_cast<float*>(smem);   // [NW][2][Nmax]
  const int t = pa.tile_begin + blockIdx.x;
  if (t >= pa.tile_end) return;
  const Tile tl = a.tiles[t];
  const GroupDev gr = a.groups[tl.group];
  const MeasRow* tab = a.table + gr.table_off;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int vl = tid / TPV, js = tid % TPV;
  const bool act = vl < tl.count;
  const int slot = tl.slot0 + vl;
  const int N = tl.n_meas;
  float th[Q];
  load_theta<K>(a.theta, a.Vpad, slot, act, th);
  Vox<K> P;
  transform<K>(th, P);
  float B = 1.f;
  if (CAL) {
    int x, y, z;
    unpack_coord(act ? a.vcoord[slot] : 0u, x, y, z);
    B = expf(tri_eval(a.gparams + gr.gp_off + 4 + 2 * gr.N4, tri_weights(x, y, z, gr.nx, gr.ny, gr.nz)));
  }
  Acc<K> A;
  acc_zero<K>(A);
  float ffin[K], fomf[K];
  fiber_weights<K>(P, ffin, fomf);
  const int iters = (N + TPV - 1) / TPV;
  for (int i = 0; i < iters; ++i) {
    const int n = i * TPV + js;
    const bool ok = act && (n < N);
    float rr = 0.f, u = 0.f;
    if (ok) {
      const size_t ix = ypos(tl, n, vl, a.VW);
      pair<K, kLossMSE, CAL, true>(P, ffin, fomf, tab[n], 0.f, B, 0.f, pa.r[ix], A, rr, u);
    }
    if (CAL) {
      float su = warp_sum_range<TPV, 16>(ok ? u : 0.f);
      float sr = warp_sum_range<TPV, 16>(ok ? rr : 0.f);
      if (lane < TPV && n < N) {
        s_ab[(warp * 2) * a.Nmax + n] = su;
        s_ab[(warp * 2 + 1) * a.Nmax + n] = sr;
      }
    }
  }
  acc_reduce_tpv<K, TPV>(A);
  float gS0, gf[NF], gd[K][3], gfin;
  data_grad<K>(P, A, 1.f, gS0, gf, gd, gfin);   // r already scaled
  float g[Q];
  chain_raw<K>(P, gS0, gf, gd, gfin, g);
  if (act && js == 0) {
#pragma unroll
    for (int q = 0; q < Q; ++q) pa.grad[static_cast<size_t>(q) * a.Vpad + slot] = g[q];
    if (CAL) a.gU[slot] = A.u;
  }
  if (CAL) {
    __syncthreads();
    const int NW = blockDim.x >> 5;
    for (int e = tid; e < 2 * N; e += blockDim.x) {
      const int w2 = (e < N) ? 0 : 1;
      const int n = e - w2 * N;
      float s = 0.f;
      for (int w = 0; w < NW; ++w) s += s_ab[(w * 2 + w2) * a.Nmax + n];
      a.tile_ab[tl.ab_off + e] = s;
    }
  }
}

// Huber-Laplacian preparation: rho'(u_c(x)) / |N(x)| and the prior value per voxel (Eq. 7).
template <int K>
__global__ void k_prior_prep(const IterArgs a, int tile_begin, int tile_end) {
  constexpr int NF = K + 3, XF = 4 * K + 3;
  // launched as a programmatic dependent of the previous iteration's fused kernel: wait for it
  // before any read, then let k_prior_grad start launching
  grid_dep_wait();
  grid_dep_launch();
  const int slot = tile_begin * a.TV + blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= tile_end * a.TV) return;
  const Tile tl = a.tiles[slot / a.TV];
  if (slot - tl.slot0 >= tl.count) return;
  const GroupDev gr = a.groups[tl.group];
  const int Vp = a.Vpad;
  const float* xf = a.xf + static_cast<size_t>((*a.step) & 1) * XF * Vp;
  const int ncnt = (a.vflag[slot] >> 8) & 31;
  float val = 0.f;
  if (ncnt == 0) {
    for (int c = 0; c < NF; ++c) a.hsp[static_cast<size_t>(c) * Vp + slot] = 0.f;
  } else {
    float sum[NF];
#pragma unroll
    for (int c = 0; c < NF; ++c) sum[c] = 0.f;
    if (a.n_nbr == 6) {
      // every index first, then every neighbour's fractions (a missing neighbour reads the
      // voxel's own row and adds nothing), so that the gathers are in flight together
      int xs[6];
#pragma unroll
      for (int e = 0; e < 6; ++e) xs[e] = a.nbr[static_cast<size_t>(e) * Vp + slot];
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const bool ok = xs[e] >= 0;
        const int x = ok ? xs[e] : slot;
#pragma unroll
        for (int c = 0; c < NF; ++c) {
          const float v = xf[static_cast<size_t>(c) * Vp + x];
          sum[c] += ok ? v : 0.f;
        }
      }
    } else {
      for (int e = 0; e < a.n_nbr; ++e) {
        const int x = a.nbr[static_cast<size_t>(e) * Vp + slot];
        if (x < 0) continue;
#pragma unroll
        for (int c = 0; c < NF; ++c) sum[c] += xf[static_cast<size_t>(c) * Vp + x];
      }
    }
    const float inv_n = 1.f / static_cast<float>(ncnt);
#pragma unroll
    for (int c = 0; c < NF; ++c) {
      const float u = xf[static_cast<size_t>(c) * Vp + slot] - sum[c] * inv_n;
      val += huber_rho(u, a.huber_delta);
      a.hsp[static_cast<size_t>(c) * Vp + slot] = huber_drho(u, a.huber_delta) * inv_n;
    }
  }
  a.lp[slot] = a.lam_sp * gr.inv_M * val;
}

// Neighbour priors of every voxel for the fused kernel (after k_prior_prep, from the current
// fractions and directions): the kPgRows<K> rows that its epilogue then reads with one
// coalesced load each instead of gathering the neighbourhood there, where the gathers'
// latency stalls the tile (on the brain workload with one thread per voxel: about 30 us here
// against 68 us of the fused kernel's epilogue).
template <int K>
__global__ void k_prior_grad(const IterArgs a, int tile_begin, int tile_end) {
  constexpr int NF = K + 3, XF = 4 * K + 3;
  // as k_prior_prep: wait for the predecessor, then let the fused kernel start launching (its
  // prologue and loop read nothing this kernel writes; it waits before its first epilogue)
  grid_dep_wait();
  grid_dep_launch();
  const int slot = tile_begin * a.TV + blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= tile_end * a.TV) return;
  const Tile tl = a.tiles[slot / a.TV];
  if (slot - tl.slot0 >= tl.count) return;
  const GroupDev gr = a.groups[tl.group];
  const int Vp = a.Vpad;
  const float* xf = a.xf + static_cast<size_t>((*a.step) & 1) * XF * Vp;
  Vox<K> P{};
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) P.d[k][c] = xf[static_cast<size_t>(K + 3 + 3 * k + c) * Vp + slot];
  float gf[NF], gd[K][3];
#pragma unroll
  for (int c = 0; c < NF; ++c) gf[c] = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) gd[k][0] = gd[k][1] = gd[k][2] = 0.f;
  const float val = nbr_priors<K>(a, P, slot, gr.inv_M, xf, gf, gd);
  float* pg = a.pg + slot;
#pragma unroll
  for (int c = 0; c < NF; ++c) pg[static_cast<size_t>(c) * Vp] = gf[c];
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int q = 0; q < 3; ++q) pg[static_cast<size_t>(NF + 3 * k + q) * Vp] = gd[k][q];
  pg[static_cast<size_t>(NF + 3 * K) * Vp] = val;
}

// Priors (and the bias-field TV term) for a tile range: value into the tile's prior
// slot (mode bit 0) and chain-ruled gradient added to `grad` / gU (mode bit 1).
template <int K>
__global__ void __launch_bounds__(256) k_prior(const IterArgs a, const PlainArgs pa) {
  constexpr int NF = K + 3, Q = 4 * K + 5, XF = 4 * K + 3;
  __shared__ double s_red[8][3];
  const int t = pa.tile_begin + blockIdx.y;
  if (t >= pa.tile_end) return;
  const Tile tl = a.tiles[t];
  const GroupDev gr = a.groups[tl.group];
  const int vl = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = vl < tl.count;
  const int slot = tl.slot0 + vl;
  const float* xf_cur = a.xf + static_cast<size_t>((*a.step) & 1) * XF * a.Vpad;
  float th[Q];
  load_theta<K>(a.theta, a.Vpad, slot, act, th);
  Vox<K> P;
  transform<K>(th, P);
  float gf[NF], gd[K][3];
#pragma unroll
  for (int i = 0; i < NF; ++i) gf[i] = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) gd[k][0] = gd[k][1] = gd[k][2] = 0.f;
  float val = 0.f;
  float gS0 = 0.f;
  if (act) {
    val = priors<K>(a, P, slot, gr.inv_M, xf_cur, gS0, gf, gd);
    if (gr.calib && a.w_tv > 0.f) {
      int x, y, z;
      unpack_coord(a.vcoord[slot], x, y, z);
      const float* blr = a.gparams + gr.gp_off + 4 + 2 * gr.N4;
      const float B0 = expf(tri_eval(blr, tri_weights(x, y, z, gr.nx, gr.ny, gr.nz)));
      float gUtv = 0.f;
      val += tv_term(blr, x, y, z, gr, a.vflag[slot], B0, a.w_tv * gr.inv_M, a.tv_eps, gUtv);
      if (pa.mode & 2) a.gU[slot] += gUtv;
    }
    if (pa.mode & 2) {
      float g[Q];
      chain_raw<K>(P, gS0, gf, gd, 0.f, g);
#pragma unroll
      for (int q = 0; q < Q; ++q) pa.grad[static_cast<size_t>(q) * a.Vpad + slot] += g[q];
    }
  }
  if (pa.mode & 1) {
    // one value per (tile, x-block): the launch uses a single x-block per tile
    double out[3];
    block_reduce3(static_cast<double>(val), 0.0, 0.0, s_red, out);
    if (threadIdx.x == 0) a.tile_red[4 * static_cast<size_t>(t) + 2] = out[0];
  }
}

}  // namespace prism
