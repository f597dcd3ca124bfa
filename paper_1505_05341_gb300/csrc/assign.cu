// Step 1 of the estimator: F = w (n - alpha n_s) on the mesh (Eq. 1; Sec. 4 assigns
// galaxies and randoms to a cubic mesh by CIC), plus the FP64 catalogue sums behind
// alpha, the normalisation I and the shot noise S (Eqs. 1 and 3).
//
// GB300 design: particles arrive in random order, and a direct global atomic
// deposit onto a 0.5-1 GB mesh would miss L2 on almost every update.  Instead a
// counting sort groups particles by mesh tile (16 x 16 x 16 nodes by default, both
// meshes of an interlaced pair held together), and one CTA per tile accumulates its
// nodes in shared memory with integer shared-memory atomics (exact fixed-point sums),
// then writes the tile with coalesced plain stores.  A particle whose stencil crosses tile borders is listed once per
// tile it touches (at most 8), so tiles never write each other's nodes: no global
// atomics on the mesh and no zero-fill pass.
//
//   k_count   : cell index per particle, FP64-accumulated sums, per-tile counts
//   k_scan    : exclusive scan of the counts (one CTA)
//   k_bin     : one 16-byte record (position, signed weight) per tile touched;
//               records whose stencils lie inside one tile fill its list from the
//               front, the others from the back, so the deposit walks the interior
//               ones without per-node range checks
//               (the deposit locates the particle again: 20-byte records with the
//               cell index cost two partial L2 sector writes each)
//   k_deposit : per-tile shared-memory deposit and store
//
// Sub-cell offsets are formed against a host-built FP64 table of node positions
// split into float (hi, lo) pairs, so d = u - floor(u) keeps ~1e-7 accuracy even
// where u = (x - box_min)/H itself is only good to ~1e-5 in float.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ys_internal.h"

namespace ys {
namespace {

constexpr int THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Cell index i and offset d in [0, 1) of coordinate x along one axis.  Returns
// false (and a periodically wrapped in-range cell) when x lies outside the box.
__device__ __forceinline__ bool locate(float x, int axis, const Geom& g, const float2* __restrict__ nodes,
                                       int& i_out, float& d_out) {
  const int n = g.n;
  const float u0 = (x - g.bmin[axis]) * g.inv_h;
  const bool finite = isfinite(u0);
  const float uc = finite ? fminf(fmaxf(u0, -2.f), (float)n + 2.f) : 0.f;
  int i = (int)floorf(uc);
  i = max(-1, min(n, i));
  const float2* nd = nodes + axis * (n + 3) + 1;  // nd[i] for i in [-1, n + 1]
  float2 nv = nd[i];
  float d = ((x - nv.x) - nv.y) * g.inv_h;
  // One-cell correction of the float guess; a particle within rounding of a node can
  // land on d = 1.0f (or a hair below 0) after it, so d is clamped into [0, 1):
  // the stencils are continuous across the node, so either side gives the same mesh.
  if (d < 0.f) {
    i = max(i - 1, -1);
    nv = nd[i];
    d = fminf(((x - nv.x) - nv.y) * g.inv_h, 0.99999994f);
  } else if (d >= 1.f) {
    i = min(i + 1, n);
    nv = nd[i];
    d = fmaxf(((x - nv.x) - nv.y) * g.inv_h, 0.f);
  }
  d = fminf(fmaxf(d, 0.f), 0.99999994f);
  const bool ok = finite && i >= 0 && i < n;
  if (!ok) {
    const float uw = finite ? u0 - floorf(u0 / (float)n) * (float)n : 0.f;
    int iw = (int)floorf(uw);
    iw = max(0, min(n - 1, iw));
    i = iw;
    d = fminf(fmaxf(uw - (float)iw, 0.f), 0.99999994f);
  }
  i_out = i;
  d_out = d;
  return ok;
}

// Stencil of one axis: up to KIND nodes and weights, for mesh 1 (nodes at i) and
// mesh 2 (nodes at i + 1/2, i.e. coordinate u - 1/2).
template <int KIND>
__device__ __forceinline__ void stencil(int i, float d, bool second, int& first, float (&w)[3]) {
  if (KIND == 1) {  // NGP
    first = second ? i : i + (d >= 0.5f ? 1 : 0);
    w[0] = 1.f;
  } else if (KIND == 2) {  // CIC
    int i2 = i;
    float d2 = d;
    if (second) {
      if (d >= 0.5f) { d2 = d - 0.5f; } else { i2 = i - 1; d2 = d + 0.5f; }
    }
    first = i2;
    w[0] = 1.f - d2;
    w[1] = d2;
  } else {  // TSC
    int c;
    float dd;
    if (second) { c = i; dd = d - 0.5f; }
    else if (d >= 0.5f) { c = i + 1; dd = d - 1.f; }
    else { c = i; dd = d; }
    first = c - 1;
    const float a = 0.5f - dd, b = 0.5f + dd;
    w[0] = 0.5f * a * a;
    w[1] = 0.75f - dd * dd;
    w[2] = 0.5f * b * b;
  }
}

// Inclusive node range [lo, hi] covered by the stencils of the M meshes.
template <int KIND, int M>
__device__ __forceinline__ void node_range(int i, float d, int& lo, int& hi) {
  float w[3];
  int f1;
  stencil<KIND>(i, d, false, f1, w);
  lo = f1;
  hi = f1 + KIND - 1;
  if (M == 2) {
    int f2;
    stencil<KIND>(i, d, true, f2, w);
    lo = min(lo, f2);
    hi = max(hi, f2 + KIND - 1);
  }
}

__device__ __forceinline__ int wrapn(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Tiles touched along one axis (1 or 2 of them).
__device__ __forceinline__ int axis_tiles(int lo, int hi, int n, int tdim, int (&t)[2]) {
  t[0] = wrapn(lo, n) / tdim;
  t[1] = wrapn(hi, n) / tdim;
  return t[0] == t[1] ? 1 : 2;
}

// HIST (counting pass only): the tile counts go to a histogram in shared memory
// (ntiles counters), added to the global counts once per CTA at the end -- a few
// CTAs per SM and a grid-stride loop, instead of one global atomic per (particle,
// tile) on counters that every SM contends for.
template <int KIND, int M, bool HIST = false, int NT = THREADS>
__global__ void __launch_bounds__(NT)
k_particles(const float* __restrict__ px, const float* __restrict__ py, const float* __restrict__ pz,
            const float* __restrict__ pw, const float* __restrict__ pnbar, int64_t n, int is_ran,
            Geom g, const float2* __restrict__ nodes, unsigned* __restrict__ tile_count,
            double* __restrict__ sums, int ntiles) {
  extern __shared__ unsigned s_hist[];
  if (HIST) {
    for (int t = threadIdx.x; t < ntiles; t += NT) s_hist[t] = 0u;
    __syncthreads();
  }
  // Compensated float sums per thread (Kahan), FP64 across threads.
  float s_w = 0.f, c_w = 0.f, s_w2 = 0.f, c_w2 = 0.f, s_w2n = 0.f, c_w2n = 0.f;
  unsigned bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // Two particles per iteration (the same order as one per iteration): their loads are issued
  // together, so that the latencies overlap.
  constexpr int U = 2;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += U * stride) {
    float xs[U], ys[U], zs[U], ws[U], nbs[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * stride < n ? base + u * stride : base;
      xs[u] = px[i];
      ys[u] = py[i];
      zs[u] = pz[i];
      ws[u] = pw ? pw[i] : 1.f;
      nbs[u] = (is_ran && pnbar) ? pnbar[i] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (base + u * stride >= n) break;
      const float x = xs[u], y = ys[u], z = zs[u], w = ws[u];
      int ci[3];
      float cd[3];
      bool ok = locate(x, 0, g, nodes, ci[0], cd[0]);
      ok &= locate(y, 1, g, nodes, ci[1], cd[1]);
      ok &= locate(z, 2, g, nodes, ci[2], cd[2]);
      int tt[3][2], nt[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        int lo, hi;
        node_range<KIND, M>(ci[a], cd[a], lo, hi);
        nt[a] = axis_tiles(lo, hi, g.n, g.tdim[a], tt[a]);
      }
      bad += ok ? 0u : 1u;
      {  // Kahan updates
        float yv = w - c_w, t = s_w + yv;
        c_w = (t - s_w) - yv; s_w = t;
        yv = w * w - c_w2; t = s_w2 + yv;
        c_w2 = (t - s_w2) - yv; s_w2 = t;
        if (is_ran && pnbar) {
          yv = w * w * nbs[u] - c_w2n; t = s_w2n + yv;
          c_w2n = (t - s_w2n) - yv; s_w2n = t;
        }
      }
      for (int a = 0; a < nt[0]; ++a)
        for (int b = 0; b < nt[1]; ++b)
          for (int c = 0; c < nt[2]; ++c) {
            const int tile = (tt[0][a] * g.tiles[1] + tt[1][b]) * g.tiles[2] + tt[2][c];
            if (HIST) atomicAdd(&s_hist[tile], 1u);
            else atomicAdd(&tile_count[tile], 1u);
          }
    }
  }
  if (HIST) {
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += NT)
      if (s_hist[t]) atomicAdd(&tile_count[t], s_hist[t]);
  }
  {
    __shared__ double red[NT / 32][4];
    double v0 = warp_sum((double)s_w - (double)c_w);
    double v1 = warp_sum((double)s_w2 - (double)c_w2);
    double v2 = warp_sum((double)s_w2n - (double)c_w2n);
    double v3 = warp_sum((double)bad);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red[wid][0] = v0; red[wid][1] = v1; red[wid][2] = v2; red[wid][3] = v3; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double t0 = 0, t1 = 0, t2 = 0, t3 = 0;
      for (int k = 0; k < NT / 32; ++k) { t0 += red[k][0]; t1 += red[k][1]; t2 += red[k][2]; t3 += red[k][3]; }
      if (is_ran) {
        atomicAdd(&sums[SUM_WR], t0);
        atomicAdd(&sums[SUM_WR2], t1);
        atomicAdd(&sums[SUM_WR2N], t2);
      } else {
        atomicAdd(&sums[SUM_WG], t0);
        atomicAdd(&sums[SUM_WG2], t1);
      }
      if (t3 != 0.0) atomicAdd(&sums[SUM_BAD], t3);
    }
  }
}

// Binning pass: one 16-byte record (position, signed weight) per tile a particle's
// stencils touch; records whose stencils lie inside one tile (no periodic wrap) fill
// the tile's list from the front (tile_cur), the others from the back (tile_back, the
// end of each list after the scan).  Each thread takes U particles per iteration, whose
// loads and first-tile cursor atomics are independent, so that their latencies
// overlap (one particle per iteration leaves the pass waiting on each memory round trip).
template <int KIND, int M, int U>
__global__ void __launch_bounds__(THREADS)
k_bin(const float* __restrict__ px, const float* __restrict__ py, const float* __restrict__ pz,
      const float* __restrict__ pw, int64_t n, int is_ran, Geom g, const float2* __restrict__ nodes,
      unsigned* __restrict__ tile_back, unsigned* __restrict__ tile_cur, float4* __restrict__ rec,
      const double* __restrict__ sums, double alpha_cfg) {
  float wscale = 1.f;
  if (is_ran) wscale = (float)(-(alpha_cfg >= 0.0 ? alpha_cfg : sums[SUM_WG] / sums[SUM_WR]));
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; base < n; base += U * stride) {
    float4 q[U];
    int tt[U][3][2], nt[U][3];
    bool inner[U], valid[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t idx = base + u * stride;
      valid[u] = idx < n;
      const int64_t i = valid[u] ? idx : base;
      q[u] = make_float4(px[i], py[i], pz[i], (pw ? pw[i] : 1.f) * wscale);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int ci[3];
      float cd[3];
      locate(q[u].x, 0, g, nodes, ci[0], cd[0]);
      locate(q[u].y, 1, g, nodes, ci[1], cd[1]);
      locate(q[u].z, 2, g, nodes, ci[2], cd[2]);
      inner[u] = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        int lo, hi;
        node_range<KIND, M>(ci[a], cd[a], lo, hi);
        nt[u][a] = axis_tiles(lo, hi, g.n, g.tdim[a], tt[u][a]);
        inner[u] = inner[u] && nt[u][a] == 1 && lo >= 0 && hi < g.n;
      }
    }
    unsigned slot[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!valid[u]) continue;
      const int tile = (tt[u][0][0] * g.tiles[1] + tt[u][1][0]) * g.tiles[2] + tt[u][2][0];
      slot[u] = inner[u] ? atomicAdd(&tile_cur[tile], 1u) : atomicSub(&tile_back[tile], 1u) - 1u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (valid[u]) rec[slot[u]] = q[u];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!valid[u] || inner[u]) continue;
      for (int a = 0; a < nt[u][0]; ++a)
        for (int b = 0; b < nt[u][1]; ++b)
          for (int c = 0; c < nt[u][2]; ++c) {
            if (a == 0 && b == 0 && c == 0) continue;  // the first tile is done
            const int tile = (tt[u][0][a] * g.tiles[1] + tt[u][1][b]) * g.tiles[2] + tt[u][2][c];
            rec[atomicSub(&tile_back[tile], 1u) - 1u] = q[u];
          }
    }
  }
}

// Exclusive scan of the tile counts (single CTA of 1024 threads); the counts are
// replaced by the end of each tile's list, the binning pass's back cursors.
__global__ void __launch_bounds__(1024)
k_scan(unsigned* __restrict__ count, int ntiles, unsigned* __restrict__ off, unsigned* __restrict__ cur) {
  __shared__ unsigned part[1024];
  const int t = threadIdx.x;
  const int per = (ntiles + 1023) / 1024;
  const int b = t * per, e = min(ntiles, b + per);
  unsigned s = 0;
  for (int i = b; i < e; ++i) s += count[i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {  // Hillis-Steele inclusive scan
    const unsigned v = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  unsigned run = t > 0 ? part[t - 1] : 0u;
  for (int i = b; i < e; ++i) {
    off[i] = run;
    cur[i] = run;
    run += count[i];
    count[i] = run;  // from here on the back cursor of tile i
  }
  if (t == 1023) off[ntiles] = part[1023];
}

// Stencil walk of one record: add(k, wxy, wz) for every node of the record's stencil,
// k the node's index in the tile's (mesh, x, y, z) order and its weight the product
// wxy * wz (wxy = wq W_x W_y, wz = W_z).  A node outside this tile goes to `trash`
// (a per-lane word past the tile that is never read): in a warp of 32 records nearly
// every stencil node is inside for some lane, so branching per node saves no adds
// and costs a divergent branch each.
template <int KIND, int M, class Add>
__device__ __forceinline__ void deposit_record(const float4& q, float wq, const Geom& g,
                                               const float2* __restrict__ nodes, const int (&o)[3],
                                               const int (&td)[3], int tvol, int trash, Add&& add) {
  const int n = g.n;
  int ci[3];
  float cd[3];  // the cell and offset the binning pass found (same arithmetic)
  locate(q.x, 0, g, nodes, ci[0], cd[0]);
  locate(q.y, 1, g, nodes, ci[1], cd[1]);
  locate(q.z, 2, g, nodes, ci[2], cd[2]);
#pragma unroll
  for (int mj = 0; mj < M; ++mj) {
    int loc[3][3];
    float wt[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int first;
      stencil<KIND>(ci[a], cd[a], mj == 1, first, wt[a]);
#pragma unroll
      for (int s = 0; s < KIND; ++s) {
        const int l = wrapn(first + s - o[a], n);  // first + s in [-1, n + 1]; o[a] in [0, n)
        loc[a][s] = (l >= 0 && l < td[a]) ? l : -1;
      }
    }
#pragma unroll
    for (int a = 0; a < KIND; ++a) {
#pragma unroll
      for (int bb = 0; bb < KIND; ++bb) {
        const float wxy = wq * wt[0][a] * wt[1][bb];
        const bool in_row = loc[0][a] >= 0 && loc[1][bb] >= 0;
        const int row = mj * tvol + (loc[0][a] * td[1] + loc[1][bb]) * td[2];
#pragma unroll
        for (int c = 0; c < KIND; ++c) add(in_row && loc[2][c] >= 0 ? row + loc[2][c] : trash, wxy, wt[2][c]);
      }
    }
  }
}

// Stencil walk of an interior record (every node of both stencils inside this tile,
// no periodic wrap): the same weights and node order as deposit_record, without the
// per-node range checks, and with the nodes of one (x, y) row at fixed offsets.
template <int KIND, int M, class Add>
__device__ __forceinline__ void deposit_inner(const float4& q, float wq, const Geom& g,
                                              const float2* __restrict__ nodes, const int (&o)[3],
                                              const int (&td)[3], int tvol, Add&& add) {
  int ci[3];
  float cd[3];
  locate(q.x, 0, g, nodes, ci[0], cd[0]);
  locate(q.y, 1, g, nodes, ci[1], cd[1]);
  locate(q.z, 2, g, nodes, ci[2], cd[2]);
#pragma unroll
  for (int mj = 0; mj < M; ++mj) {
    int first[3];
    float wt[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) stencil<KIND>(ci[a], cd[a], mj == 1, first[a], wt[a]);
    const int base = mj * tvol + ((first[0] - o[0]) * td[1] + (first[1] - o[1])) * td[2] + (first[2] - o[2]);
#pragma unroll
    for (int a = 0; a < KIND; ++a)
#pragma unroll
      for (int bb = 0; bb < KIND; ++bb) {
        const float wxy = wq * wt[0][a] * wt[1][bb];
        const int row = base + (a * td[1] + bb) * td[2];
#pragma unroll
        for (int c = 0; c < KIND; ++c) add(row + c, wxy, wt[2][c]);
      }
  }
}

// Per-tile deposit.  FIXED (the tile fits twice in shared memory): the node sums are
// kept in fixed point, as two int32 words per node, because shared-memory integer
// atomics are several times faster than float ones and integer sums are exact.
//
// Fixed point.  A node value v is stored as V = v 2^s (units of 2^-s), split into
// hi 2^sb + lo with |lo| <= 2^(sb-1); hi and lo are summed in separate int32 arrays.
// With n < 2^30 records in the tile and w_m the largest |w| among them:
//   sb = min(22, floor(31 - log2 n))  => n 2^(sb-1) <= 2^30: the lo sums cannot
//                                        overflow;
//   s  = floor(min(30 + sb - log2(n w_m), 21 + sb - log2 w_m))
//      => |V| <= 2^(21+sb) for one stencil weight (|W| <= 1), which the rounding
//         below needs, and sum |V| <= 2^(30+sb), so the hi sums stay below
//         2^30 + n/2 < 2^31.  (A float log2 off in its last bits moves these bounds by
//         a factor 1 + 1e-6, well inside the slack.)
// One stencil weight V = wxy wz 2^s (wxy already carries 2^s, an exact power-of-two
// scaling) is split without conversion instructions: fma(wxy, wz, K) with
// K = 1.5 2^(23+sb) rounds V to a multiple of 2^sb, and the bit pattern of the
// result minus that of K is V / 2^sb rounded (hi); fma(wxy, wz, -(t - K)) is the
// remainder to one float rounding, and adding 1.5 2^23 rounds it to an integer (lo).
// Each stencil weight is thus quantised to 2^-s (2^-37 of the largest weight for a
// tile of ~3000 records; 2^-17 of it for one of a million, still far finer than
// float sums, which drop every weight below half an ulp of a large node) and the sums
// are exact, so the mesh is the same bit for bit whatever order the records arrive
// in.  A tile with a non-finite weight (or 2^30 or more records) is summed in float
// instead, so that a NaN reaches exactly the nodes it touches.
//
// rmesh (shared randoms): the kept random mesh sum_ran w W, written as
// F = (galaxy deposit) - alpha rmesh, with alpha from the catalogue sums.
template <int KIND, int M, bool FIXED>
__global__ void __launch_bounds__(THREADS, 3)
k_deposit(Geom g, const float2* __restrict__ nodes, const unsigned* __restrict__ off,
          const unsigned* __restrict__ split, const float4* __restrict__ rec, float* __restrict__ mesh,
          const float* __restrict__ rmesh, const double* __restrict__ sums, double alpha_cfg) {
  extern __shared__ float s_tile[];
  __shared__ float s_wmax[THREADS / 32];
  const int n = g.n;
  const int tdx = g.tdim[0], tdy = g.tdim[1], tdz = g.tdim[2];
  const int tvol = tdx * tdy * tdz;
  const int tile = blockIdx.x;
  const int tz = tile % g.tiles[2];
  const int ty = (tile / g.tiles[2]) % g.tiles[1];
  const int tx = tile / (g.tiles[2] * g.tiles[1]);
  const int o[3] = {tx * tdx, ty * tdy, tz * tdz};
  const int td[3] = {tdx, tdy, tdz};
  const unsigned b = off[tile], e = off[tile + 1];
  const unsigned mid = split[tile];  // records [b, mid) are interior, [mid, e) cross a border
  const unsigned nrec = e - b;
  bool fixed = false;
  int sb = 0, sc = 0;  // split bits and scale exponent s
  // Layout: M tvol node words + 32 trash words, twice when FIXED (hi, then lo).
  const int words = M * tvol + 32;
  const int trash = M * tvol + (threadIdx.x & 31);
  if (FIXED) {
    for (int k = threadIdx.x; k < 2 * words; k += blockDim.x) s_tile[k] = 0.f;
    const float* wrec = reinterpret_cast<const float*>(rec) + 3;
    float wm = 0.f;
    bool bad = false;
    for (unsigned r = b + threadIdx.x; r < e; r += blockDim.x) {
      const float w = wrec[(size_t)r * 4];
      bad |= !isfinite(w);
      wm = fmaxf(wm, fabsf(w));
    }
#pragma unroll
    for (int k = 16; k > 0; k >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, k));
    if ((threadIdx.x & 31) == 0) s_wmax[threadIdx.x >> 5] = wm;
    bad = __syncthreads_or(bad);  // also orders s_wmax and the zero fill
#pragma unroll
    for (int k = 0; k < THREADS / 32; ++k) wm = fmaxf(wm, s_wmax[k]);
    fixed = !bad && nrec < (1u << 30);
    if (fixed && nrec > 0) {
      const float ln = log2f((float)nrec), lw = log2f(wm);
      sb = min(22, (int)floorf(31.f - ln));
      // s <= 100 only loses resolution; weights beyond ~2^100 (s < -100) sum in float
      const float sf = wm > 0.f ? floorf(fminf(30.f + sb - ln - lw, 21.f + sb - lw)) : 0.f;
      fixed = sf >= -100.f;
      sc = (int)fminf(100.f, fmaxf(sf, -100.f));
    }
  } else {
    for (int k = threadIdx.x; k < M * tvol; k += blockDim.x) s_tile[k] = 0.f;
    __syncthreads();
  }
  if (fixed) {
    int* s_hi = reinterpret_cast<int*>(s_tile);
    int* s_lo = s_hi + words;
    const float scale = __int_as_float((127 + sc) << 23);            // 2^s
    const int kbits = ((127 + 23 + sb) << 23) | 0x400000;            // 1.5 2^(23+sb)
    const float kh = __int_as_float(kbits);
    auto add = [&](int k, float wxy, float wz) {
      const float t = __fmaf_rn(wxy, wz, kh);
      const float lf = __fmaf_rn(wxy, wz, -__fsub_rn(t, kh));
      atomicAdd(s_hi + k, __float_as_int(t) - kbits);
      atomicAdd(s_lo + k, __float_as_int(__fadd_rn(lf, 12582912.f)) - 0x4B400000);  // + 1.5 2^23
    };
    for (unsigned r = b + threadIdx.x; r < mid; r += blockDim.x) {
      const float4 q = rec[r];
      deposit_inner<KIND, M>(q, q.w * scale, g, nodes, o, td, tvol, add);
    }
    for (unsigned r = mid + threadIdx.x; r < e; r += blockDim.x) {
      const float4 q = rec[r];
      deposit_record<KIND, M>(q, q.w * scale, g, nodes, o, td, tvol, trash, add);
    }
  } else {
    auto add = [&](int k, float wxy, float wz) { atomicAdd(s_tile + k, wxy * wz); };
    for (unsigned r = b + threadIdx.x; r < mid; r += blockDim.x) {
      const float4 q = rec[r];
      deposit_inner<KIND, M>(q, q.w, g, nodes, o, td, tvol, add);
    }
    for (unsigned r = mid + threadIdx.x; r < e; r += blockDim.x) {
      const float4 q = rec[r];
      deposit_record<KIND, M>(q, q.w, g, nodes, o, td, tvol, trash, add);
    }
  }
  __syncthreads();
  const size_t n3 = (size_t)n * n * n;
  const float ran_scale =
      rmesh ? (float)(-(alpha_cfg >= 0.0 ? alpha_cfg : sums[SUM_WG] / sums[SUM_WR])) : 0.f;
  // hi 2^sb + lo in units of 2^-s, in float: each int32 rounds to float once and the
  // fma once more (within one ulp of the exact sum, and the same bits on every run)
  const float unscale = __int_as_float((127 - sc) << 23);       // 2^-s
  const float hscale = __int_as_float((127 + sb - sc) << 23);   // 2^(sb-s)
  const int* s_hi = reinterpret_cast<const int*>(s_tile);
  // tile sides are powers of two (8, 16 or 32 for every supported mesh)
  const int shz = __ffs(tdz) - 1, shy = __ffs(tdy) - 1, shv = shz + shy + __ffs(tdx) - 1;
  for (int k = threadIdx.x; k < M * tvol; k += blockDim.x) {
    const int mj = k >> shv;
    const int lz = k & (tdz - 1);
    const int ly = (k >> shz) & (tdy - 1);
    const int lx = (k >> (shz + shy)) & (tdx - 1);
    const size_t at = mj * n3 + ((size_t)(o[0] + lx) * n + (o[1] + ly)) * n + (o[2] + lz);
    const float v = fixed ? __fmaf_rn(__int2float_rn(s_hi[k]), hscale, __int2float_rn(s_hi[words + k]) * unscale)
                          : s_tile[k];
    mesh[at] = rmesh ? fmaf(ran_scale, rmesh[at], v) : v;
  }
}

// FP64 sums of a random catalogue (sum w, sum w^2, sum w^2 nbar) for the kept copy.
__global__ void k_ran_sums(const float* __restrict__ w, const float* __restrict__ nbar, int64_t n,
                           double* __restrict__ out) {
  double s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = w ? (double)w[i] : 1.0;
    s1 += v;
    s2 += v * v;
    if (nbar) s3 += v * v * (double)nbar[i];
  }
  s1 = warp_sum(s1);
  s2 = warp_sum(s2);
  s3 = warp_sum(s3);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], s1);
    atomicAdd(&out[1], s2);
    atomicAdd(&out[2], s3);
  }
}

// rmesh != nullptr (shared randoms): ran is empty, the random sums come from rsums
// (sum w, sum w^2, sum w^2 nbar) and the deposit subtracts alpha rmesh.
// ---------------------------------------------------------------------------
// Direct assignment for meshes that stay resident in L2 (m N^3 floats of at most
// 64 MB, half of it): one pass over each catalogue adds every stencil weight
// into the zeroed mesh with global float reductions, served in L2.  The catalogue
// sums come first (the randoms carry -alpha w), so particles are read twice in all
// (4-12 bytes, then 16) instead of the sort's count, bin and deposit passes.
// ---------------------------------------------------------------------------

// Catalogue sums of Eqs. (1) and (3): Kahan-compensated float per thread, FP64
// across threads (the same slots as the sorted path's counting pass).
__global__ void __launch_bounds__(THREADS)
k_sums(const float* __restrict__ pw, const float* __restrict__ pnbar, int64_t n, int is_ran,
       double* __restrict__ sums) {
  float s_w = 0.f, c_w = 0.f, s_w2 = 0.f, c_w2 = 0.f, s_w2n = 0.f, c_w2n = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
    const float w = pw ? pw[idx] : 1.f;
    float yv = w - c_w, t = s_w + yv;
    c_w = (t - s_w) - yv; s_w = t;
    yv = w * w - c_w2; t = s_w2 + yv;
    c_w2 = (t - s_w2) - yv; s_w2 = t;
    if (is_ran && pnbar) {
      yv = w * w * pnbar[idx] - c_w2n; t = s_w2n + yv;
      c_w2n = (t - s_w2n) - yv; s_w2n = t;
    }
  }
  const double v0 = warp_sum((double)s_w - (double)c_w);
  const double v1 = warp_sum((double)s_w2 - (double)c_w2);
  const double v2 = warp_sum((double)s_w2n - (double)c_w2n);
  if ((threadIdx.x & 31) == 0) {
    if (is_ran) {
      atomicAdd(&sums[SUM_WR], v0);
      atomicAdd(&sums[SUM_WR2], v1);
      atomicAdd(&sums[SUM_WR2N], v2);
    } else {
      atomicAdd(&sums[SUM_WG], v0);
      atomicAdd(&sums[SUM_WG2], v1);
    }
  }
}

template <int KIND, int M>
__global__ void __launch_bounds__(THREADS)
k_direct(const float* __restrict__ px, const float* __restrict__ py, const float* __restrict__ pz,
         const float* __restrict__ pw, int64_t n, int is_ran, Geom g, const float2* __restrict__ nodes,
         double* __restrict__ sums, double alpha_cfg, float* __restrict__ mesh) {
  float wscale = 1.f;
  if (is_ran) wscale = (float)(-(alpha_cfg >= 0.0 ? alpha_cfg : sums[SUM_WG] / sums[SUM_WR]));
  const int nn = g.n;
  const size_t n3 = (size_t)nn * nn * nn;
  unsigned bad = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
    const float x = px[idx], y = py[idx], z = pz[idx];
    const float w = (pw ? pw[idx] : 1.f) * wscale;
    int ci[3];
    float cd[3];
    bool ok = locate(x, 0, g, nodes, ci[0], cd[0]);
    ok &= locate(y, 1, g, nodes, ci[1], cd[1]);
    ok &= locate(z, 2, g, nodes, ci[2], cd[2]);
    bad += ok ? 0u : 1u;
#pragma unroll
    for (int mj = 0; mj < M; ++mj) {
      int node[3][3];
      float wt[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        int first;
        stencil<KIND>(ci[a], cd[a], mj == 1, first, wt[a]);
#pragma unroll
        for (int s = 0; s < KIND; ++s) node[a][s] = wrapn(first + s, nn);
      }
      float* mm = mesh + mj * n3;
#pragma unroll
      for (int a = 0; a < KIND; ++a)
#pragma unroll
        for (int b = 0; b < KIND; ++b) {
          const float wxy = w * wt[0][a] * wt[1][b];
          float* row = mm + ((size_t)node[0][a] * nn + node[1][b]) * nn;
#pragma unroll
          for (int c = 0; c < KIND; ++c) atomicAdd(row + node[2][c], wxy * wt[2][c]);
        }
    }
  }
  unsigned tot = bad;  // particles outside the box
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&sums[SUM_BAD], (double)tot);
}

template <int KIND, int M>
cudaError_t run_direct(Plan& p, const ys_catalog& gal, const ys_catalog& ran) {
  cudaStream_t st = p.stream;
  cudaError_t err;
  const size_t n3 = (size_t)p.n * p.n * p.n;
  if ((err = cudaMemsetAsync(p.d_sums, 0, sizeof(double) * SUM_COUNT, st))) return err;
  if ((err = cudaMemsetAsync(p.d_mesh, 0, sizeof(float) * p.m * n3, st))) return err;
  int dev = 0, sms = 0;
  if ((err = cudaGetDevice(&dev)) || (err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
    return err;
  auto blocks = [&](int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + THREADS - 1) / THREADS, (int64_t)sms * 8));
  };
  const ys_catalog* cats[2] = {&gal, &ran};
  for (int c = 0; c < 2; ++c) {
    const ys_catalog& k = *cats[c];
    if (k.n == 0) continue;
    LaunchScope ls(p, 0);
    k_sums<<<blocks(k.n), THREADS, 0, st>>>(k.w, k.nbar, k.n, c, p.d_sums);
    if ((err = cudaGetLastError())) return err;
  }
  for (int c = 0; c < 2; ++c) {
    const ys_catalog& k = *cats[c];
    if (k.n == 0) continue;
    LaunchScope ls(p, 3);
    k_direct<KIND, M><<<blocks(k.n), THREADS, 0, st>>>(k.x, k.y, k.z, k.w, k.n, c, p.geom, p.d_nodes, p.d_sums,
                                                       p.cfg.alpha, p.d_mesh);
    if ((err = cudaGetLastError())) return err;
  }
  return cudaSuccess;
}

template <int KIND, int M>
cudaError_t run_assign(Plan& p, const ys_catalog& gal, const ys_catalog& ran, const float* rmesh = nullptr,
                       const double* rsums = nullptr) {
  cudaStream_t st = p.stream;
  cudaError_t err;
  if ((err = cudaMemsetAsync(p.d_tile_count, 0, sizeof(unsigned) * p.ntiles, st)) != cudaSuccess) return err;
  if ((err = cudaMemsetAsync(p.d_sums, 0, sizeof(double) * SUM_COUNT, st)) != cudaSuccess) return err;
  if (rsums && (err = cudaMemcpyAsync(p.d_sums + SUM_WR, rsums, sizeof(double) * 3, cudaMemcpyDeviceToDevice, st)))
    return err;
  auto blocks = [](int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + THREADS - 1) / THREADS, 152 * 16)); };
  const ys_catalog* cats[2] = {&gal, &ran};
  // counting: shared-memory histograms while the tile counters fit (a few CTAs per SM)
  constexpr int HT = 1024;
  const size_t hist_bytes = sizeof(unsigned) * (size_t)p.ntiles;
  const bool hist = hist_bytes <= 160u * 1024u;
  int hist_grid = 0;
  if (hist) {
    int dev = 0, sms = 0, per = 0;
    if ((err = cudaGetDevice(&dev)) || (err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
      return err;
    if ((err = cudaFuncSetAttribute(k_particles<KIND, M, true, HT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hist_bytes)))
      return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_particles<KIND, M, true, HT>, HT,
                                                             hist_bytes)))
      return err;
    hist_grid = std::max(1, per) * sms;
  }
  for (int c = 0; c < 2; ++c) {
    const ys_catalog& k = *cats[c];
    if (k.n == 0) continue;
    LaunchScope ls(p, 0);
    if (hist) {
      const int grid = (int)std::min<int64_t>(hist_grid, (k.n + HT - 1) / HT);
      k_particles<KIND, M, true, HT><<<grid, HT, hist_bytes, st>>>(k.x, k.y, k.z, k.w, k.nbar, k.n, c, p.geom,
                                                                  p.d_nodes, p.d_tile_count, p.d_sums, p.ntiles);
    } else {
      k_particles<KIND, M, false><<<blocks(k.n), THREADS, 0, st>>>(k.x, k.y, k.z, k.w, k.nbar, k.n, c, p.geom,
                                                                   p.d_nodes, p.d_tile_count, p.d_sums, p.ntiles);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  {
    LaunchScope ls(p, 1);
    k_scan<<<1, 1024, 0, st>>>(p.d_tile_count, p.ntiles, p.d_tile_off, p.d_tile_cur);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  for (int c = 0; c < 2; ++c) {
    const ys_catalog& k = *cats[c];
    if (k.n == 0) continue;
    LaunchScope ls(p, 2);
    constexpr int U = 2;
    k_bin<KIND, M, U><<<blocks((k.n + U - 1) / U), THREADS, 0, st>>>(
        k.x, k.y, k.z, k.w, k.n, c, p.geom, p.d_nodes, p.d_tile_count, p.d_tile_cur, p.d_rec, p.d_sums, p.cfg.alpha);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
  }
  const int tvol = p.geom.tdim[0] * p.geom.tdim[1] * p.geom.tdim[2];
  int dev = 0, optin = 0;
  if ((err = cudaGetDevice(&dev)) ||
      (err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)))
    return err;
  // fixed-point sums need two words per node; a tile that cannot hold them sums in float
  const size_t words = (size_t)M * tvol + 32;  // nodes and one trash word per lane
  const size_t smem_fixed = 2 * sizeof(float) * words;
  const bool fixed = smem_fixed + 64 <= (size_t)optin;
  const size_t smem = fixed ? smem_fixed : sizeof(float) * words;
  auto kern = fixed ? k_deposit<KIND, M, true> : k_deposit<KIND, M, false>;
  if ((err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
    return err;
  LaunchScope ls(p, 3);
  kern<<<p.ntiles, THREADS, smem, st>>>(p.geom, p.d_nodes, p.d_tile_off, p.d_tile_cur, p.d_rec, p.d_mesh, rmesh,
                                        p.d_sums, p.cfg.alpha);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_assign(Plan& p, const ys_catalog& gal, const ys_catalog& ran, const float* rmesh,
                          const double* rsums) {
  const int key = p.kind * 2 + (p.m - 1);
  if (p.direct_assign && !rmesh) {
    switch (key) {
      case 2: return run_direct<1, 1>(p, gal, ran);
      case 3: return run_direct<1, 2>(p, gal, ran);
      case 4: return run_direct<2, 1>(p, gal, ran);
      case 5: return run_direct<2, 2>(p, gal, ran);
      case 6: return run_direct<3, 1>(p, gal, ran);
      case 7: return run_direct<3, 2>(p, gal, ran);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (key) {
    case 2: return run_assign<1, 1>(p, gal, ran, rmesh, rsums);
    case 3: return run_assign<1, 2>(p, gal, ran, rmesh, rsums);
    case 4: return run_assign<2, 1>(p, gal, ran, rmesh, rsums);
    case 5: return run_assign<2, 2>(p, gal, ran, rmesh, rsums);
    case 6: return run_assign<3, 1>(p, gal, ran, rmesh, rsums);
    case 7: return run_assign<3, 2>(p, gal, ran, rmesh, rsums);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_random_sums(Plan& p, const ys_catalog& ran, double* out) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * 3, p.stream);
  if (e || ran.n == 0) return e;
  const unsigned blocks = (unsigned)std::min<int64_t>(152 * 8, (ran.n + THREADS - 1) / THREADS);
  k_ran_sums<<<blocks, THREADS, 0, p.stream>>>(ran.w, ran.nbar, ran.n, out);
  return cudaGetLastError();
}

}  // namespace ys
