// Non-templated PRISM kernels: preprocessing (b0 normalisation, packing, measurement
// tables, parameter layout), the plain-path data term and Adam, and the group-level
// reductions and updates of the calibration / noise parameters (Sec. 2.3).
#include <math.h>

#include "prism_kernels.cuh"
#include "prism_launch.h"

namespace prism {

// ---------------------------------------------------------------------------
// Preprocessing (Sec. 2.5: both y and y_hat are divided by the measured b0).
// ---------------------------------------------------------------------------
// One warp per voxel (the lanes read the row's consecutive measurements together), 256 voxels
// per block of 256 threads; part[block] is the block's sum of the squared b0 deviations. The
// per-voxel sums are FP32 (a b0 mean of a few dozen positive values, stored as FP32); the
// squared deviations accumulate in FP64 per thread and per block.
__global__ void __launch_bounds__(256) k_b0_stats(const float* __restrict__ sig, int64_t V, int N,
                                                  const uint8_t* __restrict__ isb0, int nb0,
                                                  float* __restrict__ b0mean, double* __restrict__ part, int* bad) {
  __shared__ double s[256];
  __shared__ uint8_t s_b0[1024];   // N <= 1024 (prism_fit_init checks it)
  for (int n = threadIdx.x; n < N; n += blockDim.x) s_b0[n] = isb0[n];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  for (int j = 0; j < 32; ++j) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * 256 + warp * 32 + j;
    if (v >= V) break;
    const float* row = sig + v * N;
    float m = 0.f;
    bool finite = true;
    for (int n = lane; n < N; n += 32) {
      const float x = row[n];
      if (!isfinite(x)) finite = false;
      if (s_b0[n]) m += x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
    finite = __all_sync(0xffffffffu, finite);
    m /= static_cast<float>(nb0);
    if (!finite || !(m > 0.f)) {
      if (lane == 0) atomicAdd(bad, 1);
      m = 1.f;
    }
    if (lane == 0) b0mean[v] = m;
    const float inv = 1.f / m;
    for (int n = lane; n < N; n += 32)
      if (s_b0[n]) {
        const float d = fmaf(row[n], inv, -1.f);
        acc += static_cast<double>(d * d);
      }
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// sigma init (Sec. 2.3 learns sigma but does not say where it starts): pooled std of the
// normalised b0 repeats, clamped >= 1e-3.
__global__ void k_sigma_init(const double* part, int nblocks, int64_t V, int nb0, float fallback,
                             float* sigma_log) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += part[b];
  double sg = fallback;
  if (nb0 >= 2) sg = fmax(sqrt(s / (static_cast<double>(V) * (nb0 - 1))), 1e-3);
  *sigma_log = static_cast<float>(log(sg));
}

// One tile per block of kPackThreads: each warp column of the tile (VW voxels) in chunks of
// kPackC measurements, staged in shared memory so that the reads run along the voxels' signal
// rows and the writes along the packed [pair][voxel][2] layout (ypos).
constexpr int kPackThreads = 256, kPackC = 128;
template <int VW>
__global__ void __launch_bounds__(kPackThreads) k_pack(const IterArgs a, const float* __restrict__ sig,
                                                       const float* __restrict__ b0mean,
                                                       const int32_t* __restrict__ vox_of_slot,
                                                       const int32_t* __restrict__ order, int64_t vox0, int tile_begin,
                                                       int N, float* __restrict__ ypack) {
  __shared__ float s[VW][kPackC + 1];
  __shared__ int64_t s_row[VW];   // the voxel's signal row (-1: padding slot)
  __shared__ float s_inv[VW];     // 1 / its b0 mean
  const int t = tile_begin + blockIdx.x;
  const Tile tl = a.tiles[t];
  const int NP = (N + 3) & ~3;
  for (int w = 0; w * VW < a.TV; ++w) {
    if (threadIdx.x < VW) {
      const int vl = w * VW + threadIdx.x;
      int64_t r = -1;
      float inv = 0.f;
      if (vl < tl.count) {
        const int64_t v = vox_of_slot[tl.slot0 + vl] - vox0;
        r = v * N;
        inv = 1.f / b0mean[v];
      }
      s_row[threadIdx.x] = r;
      s_inv[threadIdx.x] = inv;
    }
    __syncthreads();
    for (int n0 = 0; n0 < NP; n0 += kPackC) {
      const int C = min(kPackC, NP - n0);   // even (NP and kPackC are multiples of 4)
#pragma unroll 8
      for (int i = threadIdx.x; i < VW * C; i += kPackThreads) {
        const int j = i / C, nc = i - j * C, n = n0 + nc;
        const int64_t r = s_row[j];
        s[j][nc] = (r >= 0 && n < N) ? sig[r + order[n]] * s_inv[j] : 0.f;
      }
      __syncthreads();
      float* out = ypack + tl.y_off + static_cast<size_t>(w) * NP * VW + static_cast<size_t>(n0) * VW;
#pragma unroll 8
      for (int i = threadIdx.x; i < VW * C; i += kPackThreads) {
        const int pc = i / (2 * VW), r = i - pc * 2 * VW, j = r >> 1;
        out[i] = s[j][2 * pc + (r & 1)];
      }
      __syncthreads();
    }
  }
}

// Static part of the per-measurement table; exp(alpha) = 1, beta = 0 (identity, Sec. 2.3).
__global__ void k_table(const float* bvals, const float* bvecs, int N, MeasRow* rows) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const double b = bvals[n];
  const double L2E = 1.4426950408889634;
  const double dpar = 1.7e-3, dperp = 0.4e-3;          // Eq. 5, mm^2/s
  MeasRow r;
  r.gx = bvecs[3 * n];
  r.gy = bvecs[3 * n + 1];
  r.gz = bvecs[3 * n + 2];
  r.nkpar = static_cast<float>(-b * dpar * L2E);
  r.nkperp = static_cast<float>(-b * dperp * L2E);
  r.nkd = static_cast<float>(-b * (dpar - dperp) * L2E);
  r.ecsf = static_cast<float>(exp(-b * 3.0e-3));          // Eq. 4
  r.egm = static_cast<float>(exp(-b * 0.9e-3));
  r.eres = static_cast<float>(exp(-b * 0.2e-3));
  r.An = static_cast<float>(-2.0 * b * dpar);
  r.Bn = static_cast<float>(2.0 * b * (dperp - dpar));
  r.A = 1.f;
  r.beta = 0.f;
  r.pad0 = r.pad1 = r.pad2 = 0.f;
  rows[n] = r;
}

// Paired table of one group (MeasPair), zero past N.
__global__ void k_pair_table(const MeasRow* rows, int N, int NP, MeasPair* out) {
  const int pidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (pidx >= NP / 2) return;
  const float* r0 = reinterpret_cast<const float*>(rows + 2 * pidx);
  const bool v0 = 2 * pidx < N, v1 = 2 * pidx + 1 < N;
  float f0[16], f1[16];
  for (int f = 0; f < 16; ++f) {
    f0[f] = v0 ? r0[f] : 0.f;
    f1[f] = v1 ? r0[16 + f] : 0.f;
  }
  // field order of MeasRow: gx gy gz nkpar nkperp nkd ecsf egm eres An Bn A beta pad pad pad
  MeasPair mp;
  float* o = reinterpret_cast<float*>(&mp);
  for (int f = 0; f < 16; ++f) {
    o[2 * f] = f0[f];
    o[2 * f + 1] = f1[f];
  }
  out[pidx] = mp;
}

// Per-slot tables of one volume from its grid -> slot map (one thread per grid position):
// packed coordinates, flags (bits 0-5: the face neighbour in +x, -x, +y, -y, +z, -z is in the
// mask, any patch; bits 8-12: the count of neighbours in the same patch) and the neighbour
// slots in the same patch: the six faces first, then the edges and corners of the 3x3x3 cube
// in (i, j, k) loop order.
__global__ void k_slot_data(const Tile* __restrict__ tiles, const GroupDev* __restrict__ groups, int g,
                            const int32_t* __restrict__ slot_of_grid, int Vp, int TV, int nnb,
                            uint32_t* __restrict__ vcoord, uint32_t* __restrict__ vflag, int32_t* __restrict__ nbr) {
  const GroupDev gr = groups[g];
  const int64_t ng = static_cast<int64_t>(gr.nx) * gr.ny * gr.nz;
  const int64_t gi = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (gi >= ng) return;
  const int32_t* sog = slot_of_grid + gr.grid_off;
  const int slot = sog[gi];
  if (slot < 0) return;
  const int z = static_cast<int>(gi % gr.nz), y = static_cast<int>((gi / gr.nz) % gr.ny),
            x = static_cast<int>(gi / (static_cast<int64_t>(gr.nz) * gr.ny));
  vcoord[slot] = static_cast<uint32_t>(x) | (static_cast<uint32_t>(y) << 10) | (static_cast<uint32_t>(z) << 20);
  const int patch = tiles[slot / TV].patch;
  uint32_t fl = 0;
  int cnt = 0;
  int next = 6;   // index of the next edge / corner neighbour
  for (int pass = 0; pass < 2; ++pass)
    for (int i = -1; i <= 1; ++i)
      for (int j = -1; j <= 1; ++j)
        for (int k = -1; k <= 1; ++k) {
          const int l1 = abs(i) + abs(j) + abs(k);
          if (l1 == 0 || (pass == 0) != (l1 == 1)) continue;
          int e;
          if (pass == 0) {
            e = (i != 0) ? (i > 0 ? 0 : 1) : (j != 0) ? (j > 0 ? 2 : 3) : (k > 0 ? 4 : 5);   // +x -x +y -y +z -z
          } else {
            if (next >= nnb) continue;
            e = next++;
          }
          const int xx = x + i, yy = y + j, zz = z + k;
          if (xx < 0 || yy < 0 || zz < 0 || xx >= gr.nx || yy >= gr.ny || zz >= gr.nz) continue;
          const int sj = sog[(static_cast<int64_t>(xx) * gr.ny + yy) * gr.nz + zz];
          if (sj < 0) continue;
          if (e < 6) fl |= 1u << e;
          if (tiles[sj / TV].patch == patch) {
            nbr[static_cast<size_t>(e) * Vp + slot] = sj;
            ++cnt;
          }
        }
  vflag[slot] = fl | (static_cast<uint32_t>(cnt) << 8);
}

__global__ void k_vox_of_slot(const int32_t* __restrict__ slot_of_vox, int64_t V, int32_t* __restrict__ vox_of_slot) {
  const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (v < V) vox_of_slot[slot_of_vox[v]] = static_cast<int32_t>(v);
}

// Row gather: dst[i][:] = src[rows[i]][:] (slab volumes cut from a whole volume).
__global__ void k_gather_rows(const float* __restrict__ src, const int64_t* __restrict__ rows, int64_t n, int len,
                              float* __restrict__ dst) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= n * len) return;
  const int64_t i = e / len;
  const int c = static_cast<int>(e - i * len);
  dst[e] = src[rows[i] * len + c];
}

__global__ void k_scatter_params(const float* __restrict__ in, const int32_t* __restrict__ slot_of_vox,
                                 int64_t V, int Q, int Vpad, float* __restrict__ theta) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= V * Q) return;
  const int64_t v = e / Q;
  const int q = static_cast<int>(e - v * Q);
  theta[static_cast<size_t>(q) * Vpad + slot_of_vox[v]] = in[e];
}

__global__ void k_gather_params(const float* __restrict__ theta, const int32_t* __restrict__ slot_of_vox,
                                int64_t V, int Q, int Vpad, float* __restrict__ out) {
  const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= V * Q) return;
  const int64_t v = e / Q;
  const int q = static_cast<int>(e - v * Q);
  out[e] = theta[static_cast<size_t>(q) * Vpad + slot_of_vox[v]];
}

// Counter-based generator: splitmix64 (Steele, Lea, Flood 2014) of (seed, voxel, draw).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__device__ __forceinline__ float u01f(uint64_t h) {
  return (static_cast<float>(h >> 40) + 0.5f) * (1.f / 16777216.f);   // 24 bits, in (0, 1)
}

// Default start: S0 = 1, equal fractions, f_intra = 0.5, directions uniform on the sphere,
// drawn per grid position (so that a voxel starts from the same values whichever of the
// volume's voxels share the handle).
__global__ void k_default_init(const int32_t* __restrict__ slot_of_vox, const uint32_t* __restrict__ vcoord, int ny,
                               int nz, int64_t V, int K, int Vpad, uint64_t seed, float* __restrict__ theta) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= V) return;
  const int slot = slot_of_vox[i];
  int cx, cy, cz;
  unpack_coord(vcoord[slot], cx, cy, cz);
  const int64_t v = (static_cast<int64_t>(cx) * ny + cy) * nz + cz;
  theta[slot] = 0.5413248546129181f;   // log(e - 1): S0 = softplus(raw) = 1
  for (int i = 0; i < K + 3; ++i) theta[static_cast<size_t>(1 + i) * Vpad + slot] = 0.f;
  for (int k = 0; k < K; ++k) {
    // normalised Gaussian triple by the Box-Muller transform, in FP32 (u1 >= 2^-25 keeps the
    // radius above 2e-4, so the norm is never 0)
    float g[3];
    for (int c = 0; c < 3; c += 2) {
      const uint64_t base = seed * 0x100000001B3ull ^ (static_cast<uint64_t>(v) << 8) ^ (k * 4 + c);
      const float u1 = u01f(splitmix64(base)), u2 = u01f(splitmix64(base ^ 0xABCDEF12345ull));
      const float rad = sqrtf(-2.f * logf(u1));
      float sn, cs;
      sincospif(2.f * u2, &sn, &cs);
      g[c] = rad * cs;
      if (c + 1 < 3) g[c + 1] = rad * sn;
    }
    const float inv = rsqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    for (int c = 0; c < 3; ++c) theta[static_cast<size_t>(K + 4 + 3 * k + c) * Vpad + slot] = g[c] * inv;
  }
  theta[static_cast<size_t>(4 * K + 4) * Vpad + slot] = 0.f;
}

__global__ void k_gather_yhat(const float* __restrict__ ypack, const IterArgs a,
                              const int32_t* __restrict__ vox_of_slot, const int64_t* __restrict__ row_off,
                              const int32_t* __restrict__ order, float* __restrict__ out) {
  const Tile tl = a.tiles[blockIdx.x];
  const int32_t* ord = order + a.groups[tl.group].table_off;
  for (int e = threadIdx.x; e < tl.n_meas * a.TV; e += blockDim.x) {
    const int n = e / a.TV, vl = e - n * a.TV;
    if (vl >= tl.count) continue;
    const int64_t v = vox_of_slot[tl.slot0 + vl];
    out[row_off[v] + ord[n]] = ypack[ypos(tl, n, vl, a.VW)];
  }
}

// ---------------------------------------------------------------------------
// Plain-path data term and voxel Adam.
// ---------------------------------------------------------------------------
__global__ void k_adam_voxel(const IterArgs a, const PlainArgs pa) {
  const int slot = pa.tile_begin * a.TV + blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= pa.tile_end * a.TV) return;
  const Tile tl = a.tiles[slot / a.TV];
  if (slot - tl.slot0 >= tl.count) return;
  const float stepsz = a.adamc[0], isbc2 = a.adamc[1];
  for (int q = 0; q < a.Q; ++q) {
    const size_t ix = static_cast<size_t>(q) * a.Vpad + slot;
    const float g = pa.grad[ix];
    if (a.optimizer == 0) {
      const float mq = fmaf(a.beta1, a.m[ix], (1.f - a.beta1) * g);
      const float vq = fmaf(a.beta2, a.v[ix], (1.f - a.beta2) * g * g);
      a.m[ix] = mq;
      a.v[ix] = vq;
      a.theta[ix] -= stepsz * mq / fmaf(sqrtf(vq), isbc2, a.eps);
    } else {
      float th = a.theta[ix], mq = a.m[ix], vq = a.v[ix];
      rprop_update(th, mq, vq, g, a.lr, a.eta_minus, a.eta_plus, a.step_min, a.step_max);
      a.theta[ix] = th;
      a.m[ix] = mq;
      a.v[ix] = vq;
    }
  }
}

// ---------------------------------------------------------------------------
// Group reductions: per-tile partials -> per-group sums, fixed order (two levels:
// splits of `split_tiles` tiles, then the last-arriving block sums the splits).
// Entries: 0 data loss, 1 dJ/dsigma_log, 2 prior loss, 3.. 3+2N alpha / beta.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_group_reduce(const IterArgs a, const GroupArgs g, int what) {
  __shared__ int s_last;
  const int gi = blockIdx.z, s = blockIdx.y, ce = blockIdx.x;
  const GroupDev gr = a.groups[gi];
  const int nsplit = (gr.ntiles + g.split_tiles - 1) / g.split_tiles;
  if (s >= nsplit) return;
  const int E = 3 + ((gr.calib && (what & 2)) ? 2 * gr.N : 0);
  if (ce * 256 >= E) return;
  const int e = ce * 256 + threadIdx.x;
  const int t0 = gr.tile0 + s * g.split_tiles;
  const int t1 = min(gr.tile0 + gr.ntiles, t0 + g.split_tiles);
  double acc = 0.0;
  if (e < E) {
    if (e < 3) {
      for (int t = t0; t < t1; ++t) acc += a.tile_red[4 * static_cast<size_t>(t) + e];
    } else {
      for (int t = t0; t < t1; ++t) acc += a.tile_ab[a.tiles[t].ab_off + (e - 3)];
    }
    g.part2[static_cast<size_t>(g.split_off[gi] + s) * g.max_e + e] = acc;
  }
  __threadfence();
  __syncthreads();
  const int nce = (g.max_e + 255) / 256;
  if (threadIdx.x == 0) {
    const int prev = atomicAdd(&g.counters[gi * nce + ce], 1);
    s_last = (prev == nsplit - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (e < E) {
    double tot = 0.0;
    for (int k = 0; k < nsplit; ++k)
      tot += __ldcg(&g.part2[static_cast<size_t>(g.split_off[gi] + k) * g.max_e + e]);
    if (e == 0) {
      if (what & 1) g.gloss[gi] = tot;
    } else if (e == 1) {
      g.gred[gr.gp_off] = tot;
    } else if (e == 2) {
      if (what & 1) g.gprior[gi] = tot;
    }
    else if (e < 3 + gr.N) g.gred[gr.gp_off + 4 + (e - 3)] = tot;
    else g.gred[gr.gp_off + 4 + gr.N4 + (e - 3 - gr.N)] = tot;
  }
  if (threadIdx.x == 0) g.counters[gi * nce + ce] = 0;
}

// dJ/db_lr[c] = sum_x w_c(x) dJ/dU(x): the adjoint of the trilinear upsampling. Its weights
// factor per axis, w_c(x, y, z) = w_cx(x) w_cy(y) w_cz(z), so the sum is three contractions
// in a fixed order: over z (per (x, y) line), then y, then x; each grid voxel is read once.
// Axis weights as in tri_weights: u = clamp((i + .5) 8 / n - .5, 0, 7), i0 = min(floor u, 6),
// corner i0 takes 1 - (u - i0) and corner i0 + 1 takes u - i0.
__device__ __forceinline__ void axis_weight(int i, int n, int& i0, float& w) {
  float u = (i + 0.5f) * (8.f / n) - 0.5f;
  u = fminf(fmaxf(u, 0.f), 7.f);
  i0 = min(static_cast<int>(floorf(u)), 6);
  w = u - i0;
}

// The voxels whose weight for corner c of an n-voxel axis can be nonzero (with a margin of
// one): [lo, hi].
__device__ __forceinline__ void axis_support(int c, int n, int& lo, int& hi) {
  const float sc = n / 8.f;
  lo = (c == 0) ? 0 : max(0, static_cast<int>(floorf((c - 0.5f) * sc - 0.5f)) - 1);
  hi = (c == kGrid - 1) ? n - 1 : min(n - 1, static_cast<int>(ceilf((c + 1.5f) * sc - 0.5f)) + 1);
}
__device__ __forceinline__ float axis_corner_weight(int i, int n, int c) {
  int i0;
  float w;
  axis_weight(i, n, i0, w);
  return (c == i0) ? 1.f - w : ((c == i0 + 1) ? w : 0.f);
}

// Pass 1: G1[x][y][cz] = sum_z w_cz(z) dJ/dU(x, y, z); one warp per (x, y) line, its lanes
// strided over z, then a fixed-order butterfly over the lanes (FP32: at most 1023 terms).
__global__ void __launch_bounds__(128) k_bias_grad_z(const IterArgs a, const GroupArgs g) {
  const int gi = blockIdx.y;
  const GroupDev gr = a.groups[gi];
  const int line = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (!gr.calib || line >= gr.nx * gr.ny) return;   // warp-uniform
  double* G1 = g.bscratch + g.bs_off[2 * gi];
  float acc[kGrid];
#pragma unroll
  for (int c = 0; c < kGrid; ++c) acc[c] = 0.f;
  const int32_t* sog = g.slot_of_grid + gr.grid_off + static_cast<int64_t>(line) * gr.nz;
  for (int z = lane; z < gr.nz; z += 32) {
    const int slot = sog[z];
    if (slot < 0) continue;
    int k0;
    float wz;
    axis_weight(z, gr.nz, k0, wz);
    const float u = a.gU[slot];
#pragma unroll
    for (int c = 0; c < kGrid - 1; ++c)
      if (c == k0) {
        acc[c] = fmaf(1.f - wz, u, acc[c]);
        acc[c + 1] = fmaf(wz, u, acc[c + 1]);
      }
  }
#pragma unroll
  for (int c = 0; c < kGrid; ++c) {
    const float v = warp_sum_range<1, 16>(acc[c]);
    if (lane == 0) G1[static_cast<int64_t>(line) * kGrid + c] = v;
  }
}

// Pass 2: G2[x][cy][cz] = sum_y w_cy(y) G1[x][y][cz]; one thread per (x, cy, cz), over the
// support of cy only.
__global__ void __launch_bounds__(128) k_bias_grad_y(const IterArgs a, const GroupArgs g) {
  const int gi = blockIdx.y;
  const GroupDev gr = a.groups[gi];
  if (!gr.calib) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= gr.nx * kGrid * kGrid) return;
  const int x = e / (kGrid * kGrid), cy = (e / kGrid) % kGrid, cz = e % kGrid;
  const double* G1 = g.bscratch + g.bs_off[2 * gi];
  double* G2 = g.bscratch + g.bs_off[2 * gi + 1];
  int lo, hi;
  axis_support(cy, gr.ny, lo, hi);
  double acc = 0.0;
  for (int y = lo; y <= hi; ++y) {
    const float w = axis_corner_weight(y, gr.ny, cy);
    if (w != 0.f) acc += static_cast<double>(w) * G1[(static_cast<int64_t>(x) * gr.ny + y) * kGrid + cz];
  }
  G2[(static_cast<int64_t>(x) * kGrid + cy) * kGrid + cz] = acc;
}

// Pass 3: dJ/db_lr[cx][cy][cz] = sum_x w_cx(x) G2[x][cy][cz]; one thread per corner.
__global__ void __launch_bounds__(kNGrid) k_bias_grad_x(const IterArgs a, const GroupArgs g) {
  const int gi = blockIdx.x;
  const GroupDev gr = a.groups[gi];
  if (!gr.calib) return;
  const int c = threadIdx.x;
  const int cx = c / (kGrid * kGrid), cyz = c % (kGrid * kGrid);
  const double* G2 = g.bscratch + g.bs_off[2 * gi + 1];
  int lo, hi;
  axis_support(cx, gr.nx, lo, hi);
  double acc = 0.0;
  for (int x = lo; x <= hi; ++x) {
    const float w = axis_corner_weight(x, gr.nx, cx);
    if (w != 0.f) acc += static_cast<double>(w) * G2[static_cast<int64_t>(x) * kGrid * kGrid + cyz];
  }
  g.gred[gr.gp_off + 4 + 2 * gr.N4 + c] = acc;
}

// Group finalisation (one block): objective with the calibration regularisers of Sec. 2.4
// (L2 on alpha, beta, b_lr and TV on B; the paper gives no weights: 1e-3 each by default),
// loss history, Adam on sigma_log / alpha / beta / b_lr, table refresh, step counter.
// mode bit 0: loss; bit 1: Adam + step; bit 2: export gradients.
__global__ void __launch_bounds__(256) k_group_adam(const IterArgs a, const GroupArgs g, int mode) {
  __shared__ double s[256];
  __shared__ int s_bad, s_last;
  const int tid = threadIdx.x;
  if (tid == 0) s_bad = 0;
  const int step = *a.step;
  const float stepsz = a.adamc[0], isbc2 = a.adamc[1];
  // one block per group; the last block to finish advances the step counter
  for (int gi = blockIdx.x; gi < g.G; gi += gridDim.x) {
    const GroupDev gr = a.groups[gi];
    const int base = gr.gp_off;
    const int N = gr.N, N4 = gr.N4;
    // regulariser values
    double reg = 0.0;
    if (gr.calib) {
      for (int i = tid; i < 2 * N + kNGrid; i += blockDim.x) {
        float x;
        double w;
        if (i < N) { x = g.gparams[base + 4 + i]; w = g.w_alpha / N; }
        else if (i < 2 * N) { x = g.gparams[base + 4 + N4 + (i - N)]; w = g.w_beta / N; }
        else { x = g.gparams[base + 4 + 2 * N4 + (i - 2 * N)]; w = g.w_blr / kNGrid; }
        reg += w * static_cast<double>(x) * x;
      }
    }
    s[tid] = reg;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (tid < o) s[tid] += s[tid + o];
      __syncthreads();
    }
    if ((mode & 1) && tid == 0) {
      const double J = g.gloss[gi] + g.gprior[gi] + s[0];
      g.gloss[gi] = J;
      if (!isfinite(J)) s_bad = 1;
      if (mode & 2) g.hist[static_cast<size_t>(step % g.hist_len) * g.G + gi] = J;
    }
    __syncthreads();
    // gradients and Adam over the group's packed parameters
    const int total = 4 + 2 * N4 + kNGrid;
    for (int i = tid; i < total; i += blockDim.x) {
      float grad;
      bool train;
      const float x = g.gparams[base + i];
      if (i == 0) {
        train = (g.loss_mode == kLossNLL);
        grad = train ? static_cast<float>(g.gred[base]) : 0.f;
      } else if (i < 4) {
        train = false;
        grad = 0.f;
      } else if (i < 4 + N4) {
        train = gr.calib && (i - 4 < N);
        grad = train ? static_cast<float>(g.gred[base + i] + 2.0 * g.w_alpha / N * x) : 0.f;
      } else if (i < 4 + 2 * N4) {
        train = gr.calib && (i - 4 - N4 < N);
        grad = train ? static_cast<float>(g.gred[base + i] + 2.0 * g.w_beta / N * x) : 0.f;
      } else {
        train = gr.calib;
        grad = train ? static_cast<float>(g.gred[base + i] + 2.0 * g.w_blr / kNGrid * x) : 0.f;
      }
      if (g.gexport && (mode & 4)) g.gexport[base + i] = grad;
      if ((mode & 2) && train) {
        float mq, vq, xn = x;
        if (a.optimizer == 0) {
          mq = fmaf(a.beta1, g.gm[base + i], (1.f - a.beta1) * grad);
          vq = fmaf(a.beta2, g.gv[base + i], (1.f - a.beta2) * grad * grad);
          xn = x - stepsz * mq / fmaf(sqrtf(vq), isbc2, a.eps);
        } else {
          mq = g.gm[base + i];
          vq = g.gv[base + i];
          rprop_update(xn, mq, vq, grad, a.lr, a.eta_minus, a.eta_plus, a.step_min, a.step_max);
        }
        g.gm[base + i] = mq;
        g.gv[base + i] = vq;
        g.gparams[base + i] = xn;
        if (i >= 4 && i < 4 + 2 * N4) {
          const int n = (i < 4 + N4) ? i - 4 : i - 4 - N4;
          MeasRow* row = g.table + gr.table_off + n;
          float* pr = reinterpret_cast<float*>(g.table2 + gr.table2_off + n / 2) + (n & 1);
          if (i < 4 + N4) {
            row->A = expf(xn);
            pr[2 * kPairFieldA] = row->A;
          } else {
            row->beta = xn;
            pr[2 * kPairFieldBeta] = xn;
          }
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0 && s_bad) atomicOr(a.status, kStNonfinite);
  if (!(mode & 2)) return;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = (atomicAdd(g.gdone, 1) == static_cast<int>(gridDim.x) - 1);
  }
  __syncthreads();
  if (!s_last || tid != 0) return;
  __threadfence();
  *g.gdone = 0;
  {
    *const_cast<int32_t*>(a.step) = step + 1;
    // constants of the next iteration, t = step + 2 (bias corrections in double)
    const double t2 = static_cast<double>(step) + 2.0;
    float* ac = const_cast<float*>(a.adamc);
    ac[0] = static_cast<float>(a.lr / (1.0 - pow(static_cast<double>(a.beta1), t2)));
    ac[1] = static_cast<float>(1.0 / sqrt(1.0 - pow(static_cast<double>(a.beta2), t2)));
  }
}

// Adam constants for the coming iteration t = step + 1 (after init or a checkpoint load).
__global__ void k_adam_constants(const IterArgs a) {
  if (threadIdx.x != 0) return;
  const double t1 = static_cast<double>(*a.step) + 1.0;
  float* ac = const_cast<float*>(a.adamc);
  ac[0] = static_cast<float>(a.lr / (1.0 - pow(static_cast<double>(a.beta1), t1)));
  ac[1] = static_cast<float>(1.0 / sqrt(1.0 - pow(static_cast<double>(a.beta2), t1)));
}

// Table refresh after the caller sets group parameters (exp(alpha), beta).
__global__ void k_table_refresh(const GroupArgs g, const IterArgs a) {
  const GroupDev gr = a.groups[blockIdx.x];
  for (int n = threadIdx.x; n < gr.N; n += blockDim.x) {
    MeasRow* row = g.table + gr.table_off + n;
    row->A = gr.calib ? expf(g.gparams[gr.gp_off + 4 + n]) : 1.f;
    row->beta = gr.calib ? g.gparams[gr.gp_off + 4 + gr.N4 + n] : 0.f;
    float* pr = reinterpret_cast<float*>(g.table2 + gr.table2_off + n / 2) + (n & 1);
    pr[2 * kPairFieldA] = row->A;
    pr[2 * kPairFieldBeta] = row->beta;
  }
}

// ---------------------------------------------------------------------------
// Launchers.
// ---------------------------------------------------------------------------
static inline int nblk(int64_t n, int b) { return static_cast<int>((n + b - 1) / b); }

// The bounded-wait error path, exercised without a fault: one thread waits, with the bounded
// wait the fused kernel uses for its bulk copies, on the first phase of a fresh mbarrier that
// nothing completes (no copy is issued and nothing arrives). When the wait gives up after
// `polls` polls, the timeout bit of the status word is set and the kernel returns.
__global__ void k_wait_probe(int32_t* status, int polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (!mbar_wait(&bar, 0u, polls)) atomicOr(status, kStTimeout);
}

cudaError_t launch_wait_probe(int32_t* status, int polls, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(status, polls);
  return cudaGetLastError();
}

cudaError_t launch_group_reduce(const IterArgs& a, const GroupArgs& g, int what, cudaStream_t st) {
  dim3 grid((g.max_e + 255) / 256, g.max_split, g.G);
  k_group_reduce<<<grid, 256, 0, st>>>(a, g, what);
  return cudaGetLastError();
}
cudaError_t launch_bias_grad(const IterArgs& a, const GroupArgs& g, cudaStream_t st) {
  k_bias_grad_z<<<dim3(nblk(static_cast<int64_t>(g.max_nx) * g.max_ny, 4), g.G), 128, 0, st>>>(a, g);
  k_bias_grad_y<<<dim3(nblk(static_cast<int64_t>(g.max_nx) * kGrid * kGrid, 128), g.G), 128, 0, st>>>(a, g);
  k_bias_grad_x<<<g.G, kNGrid, 0, st>>>(a, g);
  return cudaGetLastError();
}
cudaError_t launch_group_adam(const IterArgs& a, const GroupArgs& g, int mode, cudaStream_t st) {
  k_group_adam<<<g.G, 256, 0, st>>>(a, g, mode);
  return cudaGetLastError();
}
cudaError_t launch_loss(const IterArgs& a, const PlainArgs& p, int loss, cudaStream_t st) {
  const int nt = p.tile_end - p.tile_begin;
  if (nt <= 0) return cudaSuccess;
  if (loss == kLossMSE) k_loss<kLossMSE><<<nt, 256, 0, st>>>(a, p);
  else k_loss<kLossNLL><<<nt, 256, 0, st>>>(a, p);
  return cudaGetLastError();
}
cudaError_t launch_adam_voxel(const IterArgs& a, const PlainArgs& p, cudaStream_t st) {
  const int64_t n = static_cast<int64_t>(p.tile_end - p.tile_begin) * a.TV;
  if (n <= 0) return cudaSuccess;
  k_adam_voxel<<<nblk(n, 256), 256, 0, st>>>(a, p);
  return cudaGetLastError();
}
cudaError_t launch_b0_stats(const float* sig, int64_t V, int N, const uint8_t* isb0, int nb0, float* b0mean,
                            double* part, int* bad, cudaStream_t st) {
  k_b0_stats<<<nblk(V, 256), 256, 0, st>>>(sig, V, N, isb0, nb0, b0mean, part, bad);
  return cudaGetLastError();
}
cudaError_t launch_sigma_init(const double* part, int nblocks, int64_t V, int nb0, float fb, float* out,
                              cudaStream_t st) {
  k_sigma_init<<<1, 32, 0, st>>>(part, nblocks, V, nb0, fb, out);
  return cudaGetLastError();
}
cudaError_t launch_pack(const IterArgs& a, const float* sig, const float* b0mean, const int32_t* vox_of_slot,
                        const int32_t* order, int64_t vox0, int tile_begin, int tile_end, int N, float* ypack,
                        int* bad, cudaStream_t st) {
  (void)bad;
  if (tile_end <= tile_begin) return cudaSuccess;
  if (a.TV % a.VW != 0) return cudaErrorInvalidValue;
  const int nb = tile_end - tile_begin;
  switch (a.VW) {
    case 32: k_pack<32><<<nb, kPackThreads, 0, st>>>(a, sig, b0mean, vox_of_slot, order, vox0, tile_begin, N, ypack); break;
    case 8: k_pack<8><<<nb, kPackThreads, 0, st>>>(a, sig, b0mean, vox_of_slot, order, vox0, tile_begin, N, ypack); break;
    case 2: k_pack<2><<<nb, kPackThreads, 0, st>>>(a, sig, b0mean, vox_of_slot, order, vox0, tile_begin, N, ypack); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
cudaError_t launch_slot_data(const Tile* tiles, const GroupDev* groups, int G, const GroupDev* host_groups,
                             const int32_t* slot_of_grid, const int32_t* slot_of_vox, int64_t V, int Vp, int TV, int nnb,
                             int32_t* vox_of_slot, uint32_t* vcoord, uint32_t* vflag, int32_t* nbr, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(vox_of_slot, 0xff, sizeof(int32_t) * Vp, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(vcoord, 0, sizeof(uint32_t) * Vp, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(vflag, 0, sizeof(uint32_t) * Vp, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(nbr, 0xff, sizeof(int32_t) * static_cast<size_t>(nnb) * Vp, st);
  if (e != cudaSuccess) return e;
  if (V > 0) k_vox_of_slot<<<nblk(V, 256), 256, 0, st>>>(slot_of_vox, V, vox_of_slot);
  for (int g = 0; g < G; ++g) {
    const int64_t ng = static_cast<int64_t>(host_groups[g].nx) * host_groups[g].ny * host_groups[g].nz;
    k_slot_data<<<nblk(ng, 256), 256, 0, st>>>(tiles, groups, g, slot_of_grid, Vp, TV, nnb, vcoord, vflag, nbr);
  }
  return cudaGetLastError();
}
cudaError_t launch_gather_rows(const float* src, const int64_t* rows, int64_t n, int len, float* dst,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gather_rows<<<nblk(n * len, 256), 256, 0, st>>>(src, rows, n, len, dst);
  return cudaGetLastError();
}
cudaError_t launch_table(const float* bvals, const float* bvecs, int N, MeasRow* rows, cudaStream_t st) {
  k_table<<<nblk(N, 128), 128, 0, st>>>(bvals, bvecs, N, rows);
  return cudaGetLastError();
}
cudaError_t launch_pair_table(const MeasRow* rows, int N, MeasPair* out, cudaStream_t st) {
  const int NP = (N + 3) & ~3;
  k_pair_table<<<nblk(NP / 2, 128), 128, 0, st>>>(rows, N, NP, out);
  return cudaGetLastError();
}
cudaError_t launch_scatter_params(const float* in, const int32_t* sov, int64_t V, int Q, int Vpad, float* th,
                                  cudaStream_t st) {
  if (V == 0) return cudaSuccess;
  k_scatter_params<<<nblk(V * Q, 256), 256, 0, st>>>(in, sov, V, Q, Vpad, th);
  return cudaGetLastError();
}
cudaError_t launch_gather_params(const float* th, const int32_t* sov, int64_t V, int Q, int Vpad, float* out,
                                 cudaStream_t st) {
  if (V == 0) return cudaSuccess;
  k_gather_params<<<nblk(V * Q, 256), 256, 0, st>>>(th, sov, V, Q, Vpad, out);
  return cudaGetLastError();
}
cudaError_t launch_default_init(const int32_t* sov, const uint32_t* vcoord, int ny, int nz, int64_t V, int K,
                                int Vpad, uint64_t seed, float* th, cudaStream_t st) {
  if (V == 0) return cudaSuccess;
  k_default_init<<<nblk(V, 128), 128, 0, st>>>(sov, vcoord, ny, nz, V, K, Vpad, seed, th);
  return cudaGetLastError();
}
cudaError_t launch_gather_yhat(const float* ypack, const IterArgs& a, const int32_t* vos, const int64_t* roff,
                               const int32_t* order, float* out, cudaStream_t st) {
  k_gather_yhat<<<a.ntiles, 256, 0, st>>>(ypack, a, vos, roff, order, out);
  return cudaGetLastError();
}
cudaError_t launch_adam_constants(const IterArgs& a, cudaStream_t st) {
  k_adam_constants<<<1, 32, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_table_refresh(const GroupArgs& g, const IterArgs& a, cudaStream_t st) {
  k_table_refresh<<<g.G, 128, 0, st>>>(g, a);
  return cudaGetLastError();
}

}  // namespace prism
