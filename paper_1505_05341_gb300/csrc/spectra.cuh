// Steps 2-4 of the estimator (Sec. 3, Eqs. 5-13): the line-of-sight weighted fields,
// their 3D FFTs, the k-space combination into A_0, A_2, A_4, the Legendre products
// of Eqs. (6)-(8) and the |k|-shell sums.
//
// Data flow per mesh (x-major mesh F[ix][iy][iz]):
//  k_yz (persistent, ticketed work list; see the block comment above YZParams)
//     row item     one x-plane, R rows: F and 1/|r|^2 per node, then for each pair of
//                  basis fields (F, F', F r_hat^a r_hat^b r_hat^c with c <= 1) the
//                  two real fields as one complex FFT along z, split into the two
//                  half spectra (k_z < nzc) and written to a ring slot laid out
//                  [field pair][k_z][y][2] (y contiguous, the pair's fields side by side).
//     column item  one k_z column of one plane: FFT along y of every basis field,
//                  folded with k_y, k_z polynomial weights into the groups G_{n,p}
//                  (power p of k_x; GroupTable); only the pencils (k_y, k_z) with
//                  k_y^2 + k_z^2 < n2_hi are written, layout [mesh][group][x][pencil].
//  k_x_combine  P pencils per CTA, tiles loaded by TMA: FFT along x of every group of
//             every mesh, interlacing phase and window compensation per mode, A_0
//             and k^n A_n = sum_p k_x^p G_{n,p}, then w |A_0|^2, w Re A_0 A_2^*,
//             w Re A_0 A_4^* (and w Re A_0 A_6^* for l_max = 6, the same
//             decomposition one order up) summed per shell: per-warp float bins, each with a
//             companion bin that collects the exact rounding error of every add
//             (so the pair carries the sum to ~2^-48), folded into the FP64 global
//             accumulators once per CTA.
//  k_finalize   alpha, I, S and Eqs. (6)-(8) per shell.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fft.cuh"
#include "ys_internal.h"

namespace ys {

#include "group_table.inc"

// Basis fields at the nodes.  A field is F times r_hat_x^a r_hat_y^b r_hat_z^c of
// degree d = a + b + c in {2, 4} (c <= 1), or F itself (d = 0), or F without the
// node at r = 0 (d = -1), or nothing (d = -2, past the last field).  With
// r = (X, Y, Z) from the observer, r_hat^(a,b,c) = X^a Y^b Z^c / |r|^d, and along one
// z-line X and Y are fixed: K = X^a Y^b is one number per line and field, so a node
// costs one reciprocal of |r|^2 shared by all fields plus two or three products per
// field.

// v^EXP for a small exponent 0 <= EXP <= 7, by the bits of EXP.
template <int EXP>
__device__ __forceinline__ float ipow_ct(float v) {
  const float v2 = v * v;
  float r = (EXP & 1) ? v : 1.f;
  if constexpr ((EXP & 2) != 0) r *= v2;
  if constexpr ((EXP & 4) != 0) r *= v2 * v2;
  return r;
}

// Field value at a node: f the mesh value, i2 = 1/|r|^2 (0 where r = 0), z = Z, K the
// line constant X^a Y^b; C, D the field's z power and degree (D = 2, 4 or 6 divides
// by |r|^D).  Each pair of fields is built with its exponents known at compile time.
template <int C, int D>
__device__ __forceinline__ float basis_value_ct(float f, float i2, float z, float K) {
  if constexpr (D == 0) return f;
  else if constexpr (D == -1) return i2 > 0.f ? f : 0.f;
  else if constexpr (D == -2) return 0.f;
  else {
    float v = (f * K) * i2;
    if constexpr (D >= 4) v *= i2;
    if constexpr (D == 6) v *= i2;
    if constexpr (C != 0) v *= z;
    return v;
  }
}

// ---------------------------------------------------------------------------
// y,z stage: one persistent kernel over a ticketed work list.
//
// Planes p = 0 .. m N - 1 (mesh j = p / N, x index p % N).  Per plane there are NZ
// "row items" (R rows of the plane: the basis fields, complex FFTs of two real
// fields along z, the split into the two half spectra for k_z < nzc, written to a
// ring slot laid out [field pair][k_z][y][2]) and NY = nzc "column items" (one k_z column:
// FFT along y of every basis field, the k_y, k_z polynomial fold into the k_x-power
// groups, written for the pencils of that column).  Tickets are handed out in steps:
// step t = row items of plane t, then column items of plane t - D.  Row items of
// plane p reuse ring slot p mod S once the column items of plane p - S are done;
// column items of plane p start once its row items are done.  Both waits are on
// per-plane completion counters (release / acquire), bounded in time; a CTA only
// ever waits on items claimed before its own, so the list cannot deadlock.
// ---------------------------------------------------------------------------

struct YZParams {
  const float* mesh;     // [m][N][N][N]
  const float* rel;      // [m][3][N] node - observer
  const float2* tw;      // [N]
  float2* ring;          // [S][NB][nzc][N]
  float2* gout;          // [m][NG][N][np]
  const int* col_off;    // [nzc + 1]
  int* done_z;           // [m N]
  int* done_y;           // [m N]
  int* ticket;           // [1]
  int* err;              // [1]
  int nzc, np, m, S, D;
  long long spin_limit;  // ns
  int skip_plane;        // >= 0: that plane's row items withhold their completion (test hook)
};

// Several catalogues of one configuration ("lanes", each with its own mesh, ring,
// counters, error flag and grouped output) in one launch: the ticket queue runs
// through lane 0's items, then lane 1's, and so on (end[l] = items of lanes 0..l).
// Items of different lanes never wait on each other, so the argument above holds
// lane by lane.  A single plan is the one-lane case.
struct YZMulti {
  YZParams lane[YZ_MAX_LANES];
  int end[YZ_MAX_LANES];
  int nlanes;
  int* ticket;
};


__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until *addr >= target; false (and the error flag set) on timeout
// or when another CTA has already failed.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Thread 0 waits until *addr >= target, for at most limit_ns nanoseconds; false (and
// the error flag set) on timeout, or when another CTA has already failed.
__device__ __forceinline__ bool wait_geq(const int* addr, int target, int* err, long long limit_ns) {
  const unsigned long long t0 = globaltimer_ns();
  long long it = 0;
  while (ld_acquire(addr) < target) {
    if ((++it & 31) == 0) {
      if (*reinterpret_cast<volatile int*>(err)) return false;
      if ((long long)(globaltimer_ns() - t0) > limit_ns) {
        atomicExch(err, 1);
        return false;
      }
    }
    __nanosleep(128);
  }
  return true;
}


template <int N, int ELL>
struct YZ {
  using T = GroupTable<ELL>;
  static constexpr int NB = T::NB, NG = T::NG, NPAIR = (NB + 1) / 2;
  static constexpr int E = fft_elems(N), TPL = N / E;
  static constexpr int R0 = fft_radix(N, 0);
  static constexpr int THREADS = 256;
  static constexpr int LPP = THREADS / TPL;                  // lines per pass
  static constexpr bool WARP_LOCAL = TPL <= 32;
  static constexpr int R0WS = (N >= 512 ? 8 : 16);
  static constexpr int R = (LPP > R0WS ? (LPP < N ? LPP : N) : R0WS);  // rows per row item
  static constexpr int PASSES = (R + LPP - 1) / LPP;
  static constexpr int LL = fft_line_len<N, true, (R0WS == 8)>();  // padded line length
  static constexpr size_t smem_z = sizeof(float2) * 2 * R * LL;
  static constexpr size_t smem_y = sizeof(float2) * NB * LL;
  static constexpr size_t smem_nodes = sizeof(float2) * R * N;  // (F, 1/|r|^2) per node of a row item
  static constexpr size_t smem = sizeof(float2) * N + smem_nodes + (smem_z > smem_y ? smem_z : smem_y);
  static_assert(N % R == 0, "rows per item must divide N");
  // Resident CTAs per SM the register budget is set for: two when two CTAs' shared
  // memory fits the SM (228 KB, less 1 KB reserved per CTA), else one.
  static constexpr int MIN_BLOCKS = 2 * (smem + 1024 + 64) <= 228 * 1024 ? 2 : 1;
};


// Monomial of basis field beta (its exponents a, b, c and degree d, i = 0..3) at
// compile time; fields past the last one (an odd count's partner) are zero.
template <int ELL>
__host__ __device__ constexpr int mono_ct(int beta, int i) {
  return beta < GroupTable<ELL>::NB ? GroupTable<ELL>::mono_c(beta, i) : (i == 3 ? -2 : 0);
}

// Pair PR's two basis fields at the nodes of the R rows, built with their exponents
// known at compile time, and the first FFT stage from registers into C.
template <int N, int ELL, int PR>
__device__ __forceinline__ void pair_stage0_ct(float2* C, const float2* nodes, float X, const float* __restrict__ rely,
                                               const float* __restrict__ relz, int row0) {
  using Y = YZ<N, ELL>;
  constexpr int E = Y::E, TPL = Y::TPL, R0 = Y::R0, R = Y::R, LL = Y::LL, LPP = Y::LPP;
  constexpr int FA = 2 * PR, FB = 2 * PR + 1;
  constexpr int AA = mono_ct<ELL>(FA, 0), AB = mono_ct<ELL>(FA, 1), AC = mono_ct<ELL>(FA, 2), AD = mono_ct<ELL>(FA, 3);
  constexpr int BA = mono_ct<ELL>(FB, 0), BB = mono_ct<ELL>(FB, 1), BC = mono_ct<ELL>(FB, 2), BD = mono_ct<ELL>(FB, 3);
  const int tl = threadIdx.x % TPL;
#pragma unroll
  for (int ps = 0; ps < Y::PASSES; ++ps) {
    const int row = ps * LPP + threadIdx.x / TPL;
    if (row < R) {
      const float Yc = rely[row0 + row];
      const float2* nrow = nodes + row * N;
      float2* lp = C + row * LL;
      const float Ka = ipow_ct<AA>(X) * ipow_ct<AB>(Yc), Kb = ipow_ct<BA>(X) * ipow_ct<BB>(Yc);
#pragma unroll 1
      for (int q = 0; q < E / R0; ++q) {
        float2 v[R0];
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int z = fft_in_index<N>(tl, q, r);
          const float Zc = (AC | BC) ? relz[z] : 0.f;
          const float2 fi = nrow[z];  // written by this thread in row_item
          v[r] = make_float2(basis_value_ct<AC, AD>(fi.x, fi.y, Zc, Ka), basis_value_ct<BC, BD>(fi.x, fi.y, Zc, Kb));
        }
        Dft<R0>::run(v);
        const int jq = tl + q * TPL;
        if constexpr (16 % R0 == 0) {
          float2* dst = lp + fft_pos<true>(jq * R0);  // element R0 jq + r sits r after R0 jq
#pragma unroll
          for (int r = 0; r < R0; ++r) dst[r] = v[r];
        } else {
#pragma unroll
          for (int r = 0; r < R0; ++r) lp[fft_pos<true>(jq * R0 + r)] = v[r];
        }
      }
    }
  }
}

// Run-time pair index to the compile-time build above (a uniform chain of tests).
template <int N, int ELL, int PR = 0>
__device__ __forceinline__ void pair_stage0(int pr, float2* C, const float2* nodes, float X,
                                            const float* __restrict__ rely, const float* __restrict__ relz, int row0) {
  if constexpr (PR < YZ<N, ELL>::NPAIR) {
    if (pr == PR) pair_stage0_ct<N, ELL, PR>(C, nodes, X, rely, relz, row0);
    else pair_stage0<N, ELL, PR + 1>(pr, C, nodes, X, rely, relz, row0);
  }
}

// One pair of basis fields (fa = 2 pr, fb = 2 pr + 1) for the R rows of a row item:
// fields at the nodes (first FFT stage from registers, one butterfly at a time),
// FFT along z, then the split of the two real fields into their half spectra,
// written to the ring slot.  C is one of two line buffers, so the split of this pair
// can overlap the FFT of the next.
template <int N, int ELL>
__device__ __forceinline__ void row_pair(int pr, float2* C, const float2* nodes, float X,
                                         const float* __restrict__ rely, const float* __restrict__ relz, int row0,
                                         const float2* tw, float2* __restrict__ zslot, int nzc) {
  using Y = YZ<N, ELL>;
  constexpr int TPL = Y::TPL, R = Y::R, LL = Y::LL;
  pair_stage0<N, ELL>(pr, C, nodes, X, rely, relz, row0);
  line_group_sync<TPL>();  // each line is written and read by its own threads
  FftRun<N, 1, false, true, R>::run(C, 1, LL, R, tw);
  __syncthreads();
  // Split: thread t takes row r = t mod R and k_z = t / R + i KS.  When KS is a
  // multiple of 16 the padded positions of k_z and N - k_z move by fixed steps.
  static_assert(Y::THREADS % R == 0, "split stride");
  constexpr int KS = Y::THREADS / R, PSTEP = KS / 16 * 17;
  constexpr bool STEP = KS % 16 == 0;
  const int r = threadIdx.x % R, kz0 = threadIdx.x / R;
  const float2* crow = C + r * LL;
  const float2* pk = crow + fft_pos<true>(kz0);
  const float2* pm = crow + fft_pos<true>(N - kz0);  // only read for k_z > 0
  // The ring holds the two fields of a pair side by side: one 16-byte store per node.
  float4* za = reinterpret_cast<float4*>(zslot) + ((size_t)pr * nzc + kz0) * N + row0 + r;
  for (int kz = kz0; kz < nzc; kz += KS, pk += PSTEP, pm -= PSTEP, za += (size_t)KS * N) {
    const float2 ck = STEP ? *pk : crow[fft_pos<true>(kz)];
    const float2 cm = kz ? (STEP ? *pm : crow[fft_pos<true>(N - kz)]) : ck;
    // Two real fields a + i b: A = (C_k + C_{-k}^*)/2, B = (C_k - C_{-k}^*)/(2i) (B = 0
    // past the last field).
    *za = make_float4(0.5f * (ck.x + cm.x), 0.5f * (ck.y - cm.y), 0.5f * (ck.y + cm.y), -0.5f * (ck.x - cm.x));
  }
}

// 1/x for a normal x > 0: the hardware approximation refined by one Newton-Raphson
// step, y' = y + y (1 - x y), which leaves it within about an ulp (the correctly
// rounded reciprocal costs a long instruction sequence per node).
__device__ __forceinline__ float recip_nr(float x) {
  const float y = __fdividef(1.f, x);
  return fmaf(y, fmaf(-x, y, 1.f), y);
}

// Row item: the mesh value F and 1/|r|^2 of every node of the R rows are formed once
// (each thread for the nodes it later reads, so no barrier is needed), then every
// pair of basis fields is built from them, transformed along z and split.
template <int N, int ELL>
__device__ __forceinline__ void row_item(float2* work, float2* nodes, const float* __restrict__ plane, float X,
                                         const float* __restrict__ rely, const float* __restrict__ relz, int row0,
                                         const float2* tw, float2* __restrict__ zslot, int nzc, int* ticket,
                                         int& next) {
  using Y = YZ<N, ELL>;
  constexpr int R = Y::R, LL = Y::LL, E = Y::E, TPL = Y::TPL, R0 = Y::R0, LPP = Y::LPP;
  const int tl = threadIdx.x % TPL;
#pragma unroll
  for (int ps = 0; ps < Y::PASSES; ++ps) {
    const int row = ps * LPP + threadIdx.x / TPL;
    if (row < R) {
      const float Yc = rely[row0 + row];
      const float xy2 = fmaf(X, X, Yc * Yc);
      const float* frow = plane + (size_t)(row0 + row) * N;
      float2* nrow = nodes + row * N;
#pragma unroll
      for (int q = 0; q < E / R0; ++q)
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const int z = fft_in_index<N>(tl, q, r);
          const float Zc = relz[z];
          const float r2 = fmaf(Zc, Zc, xy2);
          nrow[z] = make_float2(frow[z], r2 > 0.f ? recip_nr(r2) : 0.f);
        }
    }
  }
#pragma unroll 1
  for (int pr = 0; pr < Y::NPAIR; ++pr) {
    if (pr == Y::NPAIR - 1 && threadIdx.x == 0) next = atomicAdd(ticket, 1);  // see k_yz
    row_pair<N, ELL>(pr, work + (pr & 1) * R * LL, nodes, X, rely, relz, row0, tw, zslot, nzc);
  }
}

template <int N, int ELL>
__device__ __forceinline__ void column_fold(const float2* S, int kz, const int* __restrict__ col_off,
                                         float2* __restrict__ gout, int j, int ix, int np) {
  using Y = YZ<N, ELL>;
  constexpr int NG = Y::NG, LL = Y::LL;
  const int p0 = col_off[kz];
  const int cnt = col_off[kz + 1] - p0;
  const int kymax = (cnt - 1) / 2;
  const size_t gstep = (size_t)N * np;  // between groups
  float2* g0 = gout + ((size_t)j * NG * N + ix) * np + p0;
  // Lanes start at a multiple of 16 of the line position (k_y = -kymax sits at
  // N - kymax), so each half-warp reads 16 consecutive, 16-aligned elements.
  const int lead = (N - kymax) & 15;
  for (int q = (int)threadIdx.x - lead; q < cnt; q += blockDim.x) {
    if (q < 0) continue;
    const int ky = q - kymax;
    const float2* sp = S + fft_pos<true>(ky < 0 ? ky + N : ky);
    float2 g[NG];
    GroupTable<ELL>::combine([&](int f) { return sp[f * LL]; }, (float)ky, (float)kz, g);
    float2* gp = g0 + q;
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) gp[gi * gstep] = g[gi];
  }
}

template <int N, int ELL>
__device__ __forceinline__ void column_item(float2* S, const float2* __restrict__ zs, int nzc, int kz,
                                            const int* __restrict__ col_off, const float2* tw,
                                            float2* __restrict__ gout, int j, int ix, int np, int* ticket, int& next) {
  using Y = YZ<N, ELL>;
  constexpr int NB = Y::NB, NP = Y::NPAIR, E = Y::E, TPL = Y::TPL, R0 = Y::R0, LL = Y::LL, LPP = Y::LPP;
  const int tl = threadIdx.x % TPL;
  // One ring line holds a pair of fields (16 bytes per node): a thread group loads
  // both and runs the first FFT stage of each.
  for (int base = 0; base < NP; base += LPP) {
    const int pr = base + threadIdx.x / TPL;
    if (pr < NP) {
      const float4* line = reinterpret_cast<const float4*>(zs) + ((size_t)pr * nzc + kz) * N;
      float2 va[E], vb[E];
#pragma unroll
      for (int q = 0; q < E / R0; ++q)
#pragma unroll
        for (int r = 0; r < R0; ++r) {
          const float4 t = __ldcg(line + fft_in_index<N>(tl, q, r));
          va[q * R0 + r] = make_float2(t.x, t.y);
          vb[q * R0 + r] = make_float2(t.z, t.w);
        }
      fft_stage0_regs<N, true>(va, S + 2 * pr * LL, 1, tl);
      if (2 * pr + 1 < NB) fft_stage0_regs<N, true>(vb, S + (2 * pr + 1) * LL, 1, tl);
    }
  }
  __syncthreads();  // every ring load is done; lines 2 pr, 2 pr + 1 came from pair pr's threads
  // The ring lines of this column are dead once read: drop them from L2 without a
  // write-back (the slot is rewritten only after this item's completion is
  // released).  Each line is N * 16 bytes, a whole number of 128-byte lines.
  for (int base = 0; base < NP; base += LPP) {
    const int pr = base + threadIdx.x / TPL;
    if (pr < NP) {
      const float4* line = reinterpret_cast<const float4*>(zs) + ((size_t)pr * nzc + kz) * N;
      for (int c = tl; c < N / 8; c += TPL) asm volatile("discard.global.L2 [%0], 128;" ::"l"(line + c * 8) : "memory");
    }
  }
  FftRun<N, 1, false, true, NB>::run(S, 1, LL, NB, tw);
  __syncthreads();
  if (threadIdx.x == 0) next = atomicAdd(ticket, 1);  // see k_yz
  column_fold<N, ELL>(S, kz, col_off, gout, j, ix, np);
}

// Completion of one item: every thread's writes are ordered before thread 0's
// release-add by the barrier (the release is cumulative over them).
__device__ __forceinline__ void signal_release(int* counter) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.s32 [%0], 1;" ::"l"(counter) : "memory");
}

template <int N, int ELL>
__global__ void __launch_bounds__(256, YZ<N, ELL>::MIN_BLOCKS) k_yz(const __grid_constant__ YZMulti pm) {
  using Y = YZ<N, ELL>;
  constexpr int R = Y::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  __shared__ int s_ok;
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* nodes = tw + N;
  float2* work = nodes + (Y::smem_nodes / sizeof(float2));
  for (int k = threadIdx.x; k < N; k += blockDim.x) tw[k] = pm.lane[0].tw[k];  // same N: same twiddles
  const int NZ = N / R;
  const int total = pm.end[pm.nlanes - 1];
  const size_t n3 = (size_t)N * N * N;
  if (threadIdx.x == 0) s_item = atomicAdd(pm.ticket, 1);
  __syncthreads();
  int gitem = s_item;
  for (;;) {
    if (gitem >= total) break;
    // Thread 0 claims the next ticket shortly before this item ends (before the last
    // field pair of a row item, before the fold of a column item), so that the
    // atomic's round trip overlaps the item's tail.  A claimed item starts that
    // little later; claiming a whole item ahead delayed the items waiting on it too
    // much.  Items wait only on items of earlier tickets, so the list cannot deadlock.
    int next = -1;
    {  // L2 prefetch of the mesh rows of the row item one grid of tickets ahead
      const int ahead = gitem + (int)gridDim.x;
      if (ahead < total && threadIdx.x < R * N / 32) {
        int la = 0;
        while (ahead >= pm.end[la]) ++la;
        const YZParams& pa = pm.lane[la];
        const int ia = ahead - (la > 0 ? pm.end[la - 1] : 0);
        const int ipa = NZ + pa.nzc, sta = ia / ipa, sba = ia - sta * ipa;
        if (sba < NZ && sta < pa.m * N) {
          const int ja = sta / N, xa = sta - ja * N;
          const float* rows = pa.mesh + ja * n3 + (size_t)xa * N * N + (size_t)sba * R * N;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(rows + threadIdx.x * 32));  // one 128-byte line each
        }
      }
    }
    int l = 0;
    while (gitem >= pm.end[l]) ++l;
    const YZParams& prm = pm.lane[l];
    const int item = gitem - (l > 0 ? pm.end[l - 1] : 0);
    const int NY = prm.nzc, IPS = NZ + NY;
    const int mN = prm.m * N;
    const size_t slot_elems = (size_t)2 * Y::NPAIR * prm.nzc * N;  // float2 units, field pairs interleaved
    const int step = item / IPS, sub = item - step * IPS;
    if (sub < NZ) {
      const int p = step;  // row item of plane p
      if (p < mN) {
        if (threadIdx.x == 0)
          s_ok = (p < prm.S) ? 1 : (int)wait_geq(prm.done_y + (p - prm.S), NY, prm.err, prm.spin_limit);
        __syncthreads();
        if (!s_ok) break;
        const int j = p / N, ix = p - j * N;
        const float* rel = prm.rel + (size_t)j * 3 * N;
        row_item<N, ELL>(work, nodes, prm.mesh + j * n3 + (size_t)ix * N * N, rel[ix], rel + N, rel + 2 * N, sub * R,
                         tw, prm.ring + (size_t)(p % prm.S) * slot_elems, prm.nzc, pm.ticket, next);
        if (p != prm.skip_plane) signal_release(prm.done_z + p);
        else __syncthreads();  // withheld: the column items of plane p wait until their limit
      }
    } else {
      const int p = step - prm.D;  // column item of plane p
      if (p >= 0) {
        if (threadIdx.x == 0) s_ok = (int)wait_geq(prm.done_z + p, NZ, prm.err, prm.spin_limit);
        __syncthreads();
        if (!s_ok) break;
        const int j = p / N, ix = p - j * N;
        column_item<N, ELL>(work, prm.ring + (size_t)(p % prm.S) * slot_elems, prm.nzc, sub - NZ, prm.col_off, tw,
                            prm.gout, j, ix, prm.np, pm.ticket, next);
        signal_release(prm.done_y + p);
      }
    }
    __syncthreads();  // every thread is past this item before s_item changes
    if (threadIdx.x == 0) s_item = next >= 0 ? next : atomicAdd(pm.ticket, 1);
    __syncthreads();
    gitem = s_item;
  }
}


// The x stage of several lanes (catalogues of one configuration, as for k_yz) in one
// launch: grid (blocks per lane, lanes); the tables (pencils, twiddles, window, phases,
// shell lookup) are the configuration's and the same for every lane.
struct XMulti {
  CUtensorMap map[YZ_MAX_LANES];
  double* acc[YZ_MAX_LANES];
  int* err[YZ_MAX_LANES];
  int nlanes;
};

// First group of the multipole that group g belongs to (groups: A_0 | l = 2, powers
// 0..2 of k_x | l = 4, powers 0..4 | l = 6, powers 0..6), and its last.
__host__ __device__ constexpr int group_first(int g) { return g == 0 ? 0 : (g <= 3 ? 1 : (g <= 8 ? 4 : 9)); }
__host__ __device__ constexpr int group_last(int g) { return g == 0 ? 0 : (g <= 3 ? 3 : (g <= 8 ? 8 : 15)); }

// Group transformed at tile position q of a pencil block.  With HORNER the powers of
// k_x of each multipole come highest first, so that the x stage can sum them by
// Horner's rule (see k_x_combine); otherwise in table order.
template <bool HORNER>
__host__ __device__ constexpr int tile_group(int q) {
  return HORNER ? group_first(q) + group_last(q) - q : q;
}

// Whether the x stage sums the k_x powers of each multipole by the compensated
// Horner scheme (see k_x_combine): always for l_max = 6, and for l_max = 2, 4 except
// at 256^3 and 512^3, where the x stage is held to 80 registers for three CTAs per SM
// and the extra error terms would spill (shells there hold many modes, and the
// plain sums meet the parity bar with a wide margin).
template <int N, int ELL>
__host__ __device__ constexpr bool x_horner() { return ELL == 6 || (ELL >= 2 && N != 256 && N != 512); }

// ---------------------------------------------------------------------------
// x stage: FFT along x of every (mesh, group) tile of P pencils, fed by TMA.
// The grouped y,z transforms are a 2D tensor [m NG N rows][np_pad pencils] of
// float2; one tile (all N rows x P pencils) arrives by BOXES 2D bulk-tensor copies
// into one of two shared buffers (mbarrier completion), so the copy of the next
// tile overlaps the FFT of this one.  The last FFT stage stays in registers: each
// thread owns E modes (one pencil, E values of k_x) for the whole pencil block and
// accumulates A_0 and k^n A_n there; the per-mode terms of the shell sums go to
// compensated per-warp float bins in shared memory (add_compensated), folded into
// the FP64 accumulators when the CTA ends.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait for the given phase parity of an mbarrier; false on timeout.
// Wait for an mbarrier phase for at most limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit_ns) {
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((long long)(globaltimer_ns() - t0) > limit_ns) return false;
  }
}

// Exact rounding error (a + b) - fl(a + b) of a float add (Knuth's TwoSum).
// The shell bins use it with shared-memory atomics: the atomic returns the value it
// added to, so the stored sum is fl(old + v), and two_sum_err(old, v) is the exact
// error of that add whatever other threads add before or after; it goes into a
// companion bin.  Summed over every add, sum + companion equals the exact sum up to
// the companion's own rounding, a relative ~2^-24 of the errors themselves: the pair
// accumulates like FP64 on the FP32 pipes (FP64 arithmetic on this GPU runs at a
// small fraction of FP32).  The atomic flushes a subnormal sum to zero; that changes
// the error by less than 2^-126.
__device__ __forceinline__ float two_sum_err(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return (a - (s - bb)) + (b - bb);
}

template <int N, int ELL, int M, int PX = k3_pencils(N)>
struct XCombine {
  static constexpr int P = PX;  // pencils per CTA
  static constexpr int E = fft_elems_lf(N);
  static constexpr int TPL = N / E;
  static constexpr int THREADS = P * TPL;
  static constexpr int NW = THREADS / 32;
  static constexpr int NG = GroupTable<ELL>::NG;
  // shell-sum slots: |A_0|^2, Re A_0 A_2^*, Re A_0 A_4^* (and Re A_0 A_6^* for l = 6)
  static constexpr int SLOTS = ELL == 6 ? 4 : 3;
  static constexpr int TILES = NG * M;
  static constexpr int BOX_ROWS = x_box_rows(N);
  static constexpr int BOXES = N / BOX_ROWS;
  static_assert(BOXES * BOX_ROWS == N, "boxes must tile the x axis");
  static constexpr unsigned TILE_BYTES = (unsigned)(N * P * sizeof(float2));
  // work buffer padded (lf_pad) where the first stage is radix 8
  static constexpr int PADW = fft_radix(N, 0) == 8 ? P : 0;
  static constexpr int WK_ELEMS = lf_pad<PADW>(N * P);
  static constexpr int RL = fft_radix(N, fft_nstages(N) - 1);  // last radix
  // resident CTAs per SM the register budget is set for (3 x 256 threads at 256^3, 512^3)
  static constexpr int MIN_BLOCKS = ((N == 256 || N == 512) && ELL <= 4 && THREADS == 256) ? 3 : 1;
  static_assert(THREADS % 32 == 0, "threads");
  // nwb copies of the compensated float shell bins: a sum and an error term per shell
  // and slot.  With nwb = NW c (c copies per warp) lane l = p + P j of warp w adds into
  // copy w c + j mod c, which divides the lanes of one pencil (neighbouring k_x, mostly
  // one shell) that would hit one address in one instruction (same-address shared
  // atomics are served one after another); with fewer copies warp w adds into copy
  // w mod nwb.
  static size_t smem(int nbins, int nwb) {
    size_t b = 2 * (size_t)TILE_BYTES + sizeof(float2) * WK_ELEMS;  // two tile buffers and a work buffer
    b += sizeof(float2) * 2 * N + sizeof(float) * N;         // twiddles, phases, windows
    b += sizeof(float) * 2 * nwb * SLOTS * nbins;            // float bins and their error terms
    return b + 128;                                          // alignment slack
  }
};

template <int N, int ELL, int M, int PX>
__global__ void __launch_bounds__(XCombine<N, ELL, M, PX>::THREADS, XCombine<N, ELL, M, PX>::MIN_BLOCKS)
k_x_combine(const __grid_constant__ XMulti pm, int np_pad, const short2* __restrict__ pencil,
            const float2* __restrict__ tw_g, const float* __restrict__ invw_g, const float2* __restrict__ phase_g,
            const short* __restrict__ lut, int n2_hi, int nbins, int nwb) {
  // lane blockIdx.y: its grouped transforms (tensor map), shell accumulators, error flag
  const CUtensorMap* gmap = &pm.map[blockIdx.y];
  double* __restrict__ acc = pm.acc[blockIdx.y];
  int* __restrict__ err = pm.err[blockIdx.y];
  using XC = XCombine<N, ELL, M, PX>;
  constexpr int P = XC::P, E = XC::E, TPL = XC::TPL, TILES = XC::TILES, RL = XC::RL;
  constexpr bool HORNER = x_horner<N, ELL>();
  constexpr int NBL = E / RL;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar[2];
  __shared__ int s_fail;
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float2* T0 = reinterpret_cast<float2*>(base);
  float2* Wk = T0 + 2 * N * P;  // second buffer of the out-of-place stages (padded)
  float2* tw = Wk + XC::WK_ELEMS;
  float2* phs = tw + N;
  float* invw = reinterpret_cast<float*>(phs + N);
  constexpr int SLOTS = XC::SLOTS;
  float* wbin = invw + N;                    // [nwb][SLOTS][nbins] sums
  float* wcmp = wbin + nwb * SLOTS * nbins;  // [nwb][SLOTS][nbins] their rounding errors
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int k = tid; k < N; k += blockDim.x) {
    tw[k] = tw_g[k];
    phs[k] = phase_g[k];
    invw[k] = invw_g[k];
  }
  for (int k = tid; k < 2 * nwb * SLOTS * nbins; k += blockDim.x) wbin[k] = 0.f;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int npb = np_pad / P;
  const int mine = blockIdx.x < npb ? (npb - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int total = mine * TILES;
  auto issue = [&](int s) {
    const int k = s / TILES, t = s - k * TILES;
    const int gi = tile_group<HORNER>(t / M), mj = t - (t / M) * M;
    const int pb = blockIdx.x + k * gridDim.x;
    float2* dst = T0 + (s & 1) * N * P;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[s & 1], XC::TILE_BYTES);
#pragma unroll
    for (int bx = 0; bx < XC::BOXES; ++bx)
      tma_load_2d(dst + bx * XC::BOX_ROWS * P, gmap, pb * P * 2, (mj * XC::NG + gi) * N + bx * XC::BOX_ROWS, &bar[s & 1]);
  };
  if (tid == 0 && total > 0) issue(0);
  const int p = tid % P, tl = tid / P;
  float2 a0[E], ga[E];
  float2 gl[HORNER ? E : 1];  // rounding errors of the Horner sums in ga
  int bins[E];  // shell of each of this thread's modes in the current pencil (-1: none)
  int ky = 0, kz = -1, iyk = 0;
  float cf_pen = 0.f;
  float2 ph_pen = make_float2(1.f, 0.f);
  int s_stop = total;  // step whose wait ran out (copies s_stop and s_stop + 1 may be in flight)
  for (int s = 0; s < total; ++s) {
    if (tid == 0 && s + 1 < total) issue(s + 1);
    if (!mbar_wait(&bar[s & 1], (s >> 1) & 1, 1000000000LL)) s_fail = 1;  // 1 s
    __syncthreads();
    if (s_fail) {
      s_stop = s;
      break;
    }
    const int k = s / TILES, t = s - k * TILES;
    const int gi = tile_group<HORNER>(t / M), mj = t - (t / M) * M;
    if (t == 0) {
      const short2 pc = pencil[(blockIdx.x + k * gridDim.x) * P + p];
      ky = pc.x;
      kz = pc.y;
      iyk = ky < 0 ? ky + N : ky;
      const int kzc = kz < 0 ? 0 : kz;
      cf_pen = invw[iyk] * invw[kzc] * (M == 2 ? 0.5f : 1.f);
      ph_pen = cmul(phs[iyk], phs[kzc]);
#pragma unroll
      for (int q = 0; q < NBL; ++q)
#pragma unroll
        for (int r = 0; r < RL; ++r) {
          const int kx = tl + q * TPL + r * (N / RL);
          const int mx = kx <= N / 2 ? kx : kx - N;
          const int n2 = mx * mx + ky * ky + kz * kz;
          bins[q * RL + r] = (kz >= 0 && n2 < n2_hi) ? lut[n2] : -1;
        }
    }
    float2* Tb = T0 + (s & 1) * N * P;
    constexpr int SM_STAGES = fft_nstages(N) - 1;  // stages through shared memory
    FftPingPong<N, 0, SM_STAGES, 0, XC::PADW>::run(Tb, Wk, P, 1, P, tw);
    const float2* Tf = (SM_STAGES % 2 == 0) ? Tb : Wk;
    constexpr int PADF = (SM_STAGES % 2 == 0) ? 0 : XC::PADW;
    float2 v[E];
    fft_last_stage_regs<N, true, false, PADF>(Tf, p, P, tl, tw, v);
    const int first = group_first(gi);
    const int pw = gi - first;  // power of k_x
#pragma unroll
    for (int q = 0; q < NBL; ++q)
#pragma unroll
      for (int r = 0; r < RL; ++r) {
        const int e = q * RL + r;
        const int kx = tl + q * TPL + r * (N / RL);
        const int mx = kx <= N / 2 ? kx : kx - N;
        float2 X = v[e];
        if (M == 2 && mj == 1) X = cmul(X, cmul(phs[kx], ph_pen));
        if (HORNER && gi != 0) {
          // sum_p m_x^p X_p by Horner's rule (highest power first), every step
          // error-free: the product by the integer m_x is split exactly with an FMA
          // and the add with TwoSum, and both errors go to gl.  The window and the
          // interlacing mean, common to all powers, are applied at completion.
          if (mj == 0 && gi == group_last(gi)) {
            ga[e] = X;
            gl[e] = make_float2(0.f, 0.f);
          } else {
            const float m = mj == 0 ? (float)mx : 1.f;
            const float pr = ga[e].x * m, pi = ga[e].y * m;
            const float er = fmaf(ga[e].x, m, -pr), ei = fmaf(ga[e].y, m, -pi);
            ga[e].x = pr + X.x;
            ga[e].y = pi + X.y;
            gl[e].x = fmaf(gl[e].x, m, er) + two_sum_err(pr, X.x);
            gl[e].y = fmaf(gl[e].y, m, ei) + two_sum_err(pi, X.y);
          }
          continue;
        }
        float kp = cf_pen * invw[kx];
        for (int u = 0; u < pw; ++u) kp *= (float)mx;
        if (gi == 0) {
          if (mj == 0) a0[e] = make_float2(kp * X.x, kp * X.y);
          else { a0[e].x = fmaf(kp, X.x, a0[e].x); a0[e].y = fmaf(kp, X.y, a0[e].y); }
        } else if (gi == first && mj == 0) {
          ga[e] = make_float2(kp * X.x, kp * X.y);
        } else {
          ga[e].x = fmaf(kp, X.x, ga[e].x);
          ga[e].y = fmaf(kp, X.y, ga[e].y);
        }
      }
    // a multipole is complete after its last tile (for l = 6 its power-0 group)
    const bool complete = (mj == M - 1) && (HORNER ? gi == group_first(gi) : gi == group_last(gi));
    if (complete) {
      const int slot = gi == 0 ? 0 : (gi <= 3 ? 1 : (gi <= 8 ? 2 : 3));
      if (HORNER && slot > 0) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int kx = tl + (e / RL) * TPL + (e % RL) * (N / RL);
          const float c = cf_pen * invw[kx];
          ga[e] = make_float2(c * (ga[e].x + gl[e].x), c * (ga[e].y + gl[e].y));
        }
      }
      // the lanes of one pencil (lane = p + P j) hold neighbouring k_x, mostly in one
      // shell: spread them over the warp's copies by j
      const int copy = nwb >= XC::NW ? warp * (nwb / XC::NW) + ((tid & 31) / P) % (nwb / XC::NW) : warp % nwb;
      float* wb = wbin + (copy * SLOTS + slot) * nbins;
      float* wc = wb + nwb * SLOTS * nbins;
      const float wgt = kz == 0 ? 1.f : 2.f;
      // The lanes of one pencil (lane = p + P j, j < 32 / P) hold neighbouring k_x and
      // mostly share a shell: each run of equal shells (cut wherever neighbouring lanes
      // differ) is first summed across its lanes by a segmented suffix scan with
      // compensated adds, and only the run's first lane adds it to the bins.
      const int lane = tid & 31, jl = lane / P;
      constexpr int LG = 32 / P;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int kx = tl + (e / RL) * TPL + (e % RL) * (N / RL);
        const int mx = kx <= N / 2 ? kx : kx - N;
        float val;
        if (slot == 0) {
          val = wgt * (a0[e].x * a0[e].x + a0[e].y * a0[e].y);
        } else {
          const float inv = 1.f / (float)(mx * mx + ky * ky + kz * kz);
          const float ik = slot == 1 ? inv : (slot == 2 ? inv * inv : inv * inv * inv);  // 1 / k^(2 slot)
          val = wgt * ik * (a0[e].x * ga[e].x + a0[e].y * ga[e].y);
        }
        const int key = bins[e];
        const int key_next = __shfl_down_sync(0xffffffffu, key, P);
        const int key_prev = __shfl_up_sync(0xffffffffu, key, P);
        int end = (jl == LG - 1 || key_next != key) ? 1 : 0;  // this lane's run stops here
        float cmp = 0.f;
#pragma unroll
        for (int d = P; d < 32; d <<= 1) {
          const float vn = __shfl_down_sync(0xffffffffu, val, d);
          const float cn = __shfl_down_sync(0xffffffffu, cmp, d);
          const int en = __shfl_down_sync(0xffffffffu, end, d);
          if (!end) {  // the run reaches lane + d, inside this pencil's lanes
            cmp += cn + two_sum_err(val, vn);
            val += vn;
            end = en;
          }
        }
        if (key >= 0 && (jl == 0 || key_prev != key)) {
          const float old = atomicAdd(wb + key, val);
          const float err = cmp + two_sum_err(old, val);
          if (err != 0.f) atomicAdd(wc + key, err);
        }
      }
    }
    __syncthreads();
  }
  if (s_fail) {
    if (tid == 0) {
      atomicExch(err, 2);
      // Copies s_stop and s_stop + 1 (if issued) are the last ones issued into their
      // buffers: wait for each by its own phase parity before the CTA's shared memory
      // is released (bounded; every earlier copy has completed).
      for (int s = s_stop; s < s_stop + 2 && s < total; ++s) mbar_wait(&bar[s & 1], (s >> 1) & 1, 100000000LL);
    }
    return;
  }
  // FP64 fold of every warp copy's sum and error term, once per CTA.
  for (int b = tid; b < SLOTS * nbins; b += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < nwb; ++w) v += (double)wbin[w * SLOTS * nbins + b] + (double)wcmp[w * SLOTS * nbins + b];
    if (v != 0.0) atomicAdd(&acc[b], v);
  }
}

}  // namespace ys
