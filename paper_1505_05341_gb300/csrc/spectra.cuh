// Steps 2-4 of the estimator (Sec. 3, Eqs. 5-13): the line-of-sight weighted fields,
// their 3D FFTs, the k-space combination into A_0, A_2, A_4, the Legendre products
// of Eqs. (6)-(8) and the |k|-shell sums.
//
// Data flow per mesh (x-major mesh F[ix][iy][iz]):
//  k_yz_rows  one x-plane, R rows per CTA: builds the basis fields F, F', and
//             F r_hat^a r_hat^b r_hat^c (c <= 1) at the nodes, two real fields per
//             complex row FFT along z, splits the pair into the two half spectra
//             (k_z <= k_z,max) and writes them to a scratch laid out [field][plane]
//             [k_z][y] (y contiguous).
//  k_yz_cols  one x-plane, KC k_z columns per CTA: FFT along y of every basis field,
//             then folds them with k_y, k_z polynomial weights into the groups
//             G_{n,p} (power p of k_x; GroupTable) and writes only the pencils
//             (k_y, k_z) with k_y^2 + k_z^2 < n2_hi, layout [mesh][group][x][pencil].
//  k_x_combine  P pencils per CTA: FFT along x of every group of every mesh,
//             interlacing phase and window compensation per mode, A_0 and
//             k^n A_n = sum_p k_x^p G_{n,p}, then w |A_0|^2, w Re A_0 A_2^*,
//             w Re A_0 A_4^* summed per shell (warp segmented sums in float, FP64
//             shared and global accumulators).
//  k_finalize   alpha, I, S and Eqs. (6)-(8) per shell.
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"
#include "ys_internal.h"

namespace ys {

#include "group_table.inc"

// Rows per CTA in k_yz_rows and pencils per CTA in k_x_combine.
constexpr int KZ_ROWS = 16;
constexpr int KZ_THREADS = 256;
constexpr int KY_THREADS = 256;

template <int A>
__device__ __forceinline__ float ipow(float v) {
  float r = 1.f;
#pragma unroll
  for (int i = 0; i < A; ++i) r *= v;
  return r;
}

// Value of basis field `beta` at one node.
template <int ELL, int BETA>
__device__ __forceinline__ float basis_value(float f, float xh, float yh, float zh, bool nonzero_r) {
  using T = GroupTable<ELL>;
  if constexpr (BETA >= T::NB) {
    return 0.f;
  } else {
    constexpr int a = T::MONO[BETA][0], b = T::MONO[BETA][1], c = T::MONO[BETA][2], d = T::MONO[BETA][3];
    if constexpr (d == 0) return f;
    else if constexpr (d == -1) return nonzero_r ? f : 0.f;
    else return f * ipow<a>(xh) * ipow<b>(yh) * ipow<c>(zh);
  }
}

template <int N, int ELL, int PAIR>
__device__ __forceinline__ void fill_pair(float2* C, const float* Fs, float X, const float* __restrict__ rely,
                                          const float* __restrict__ relz, int row0) {
  for (int e = threadIdx.x; e < KZ_ROWS * N; e += blockDim.x) {
    const int r = e / N, z = e - (e / N) * N;
    const float Y = rely[row0 + r], Z = relz[z];
    const float f = Fs[e];
    const float r2 = fmaf(X, X, fmaf(Y, Y, Z * Z));
    const bool nz = r2 > 0.f;
    const float rinv = nz ? rsqrtf(r2) : 0.f;
    const float xh = X * rinv, yh = Y * rinv, zh = Z * rinv;
    C[r * (N + 1) + z] = make_float2(basis_value<ELL, 2 * PAIR>(f, xh, yh, zh, nz),
                                     basis_value<ELL, 2 * PAIR + 1>(f, xh, yh, zh, nz));
  }
}

template <int N, int ELL, int PAIR>
__device__ __forceinline__ void split_store(const float2* C, float2* __restrict__ zbuf, int slot, int batch,
                                            int nzc, int row0) {
  constexpr int NB = GroupTable<ELL>::NB;
  constexpr int FA = 2 * PAIR, FB = 2 * PAIR + 1;
  for (int e = threadIdx.x; e < nzc * KZ_ROWS; e += blockDim.x) {
    const int kz = e / KZ_ROWS, r = e - kz * KZ_ROWS;
    const float2 ck = C[r * (N + 1) + kz];
    const float2 cm = C[r * (N + 1) + (kz == 0 ? 0 : N - kz)];
    // Two real fields a + i b: A = (C_k + C_{-k}^*)/2, B = (C_k - C_{-k}^*)/(2i).
    const float2 A = make_float2(0.5f * (ck.x + cm.x), 0.5f * (ck.y - cm.y));
    zbuf[(((size_t)FA * batch + slot) * nzc + kz) * N + row0 + r] = A;
    if constexpr (FB < NB) {
      const float2 B = make_float2(0.5f * (ck.y + cm.y), -0.5f * (ck.x - cm.x));
      zbuf[(((size_t)FB * batch + slot) * nzc + kz) * N + row0 + r] = B;
    }
  }
}

template <int N, int ELL, int PAIR>
struct PairLoop {
  __device__ static __forceinline__ void run(float2* C, const float* Fs, float X, const float* rely,
                                             const float* relz, int row0, const float2* tw, float2* zbuf,
                                             int slot, int batch, int nzc) {
    constexpr int NB = GroupTable<ELL>::NB;
    if constexpr (2 * PAIR < NB) {
      fill_pair<N, ELL, PAIR>(C, Fs, X, rely, relz, row0);
      __syncthreads();
      fft_smem<N, false>(C, 1, N + 1, KZ_ROWS, tw);
      split_store<N, ELL, PAIR>(C, zbuf, slot, batch, nzc, row0);
      __syncthreads();
      PairLoop<N, ELL, PAIR + 1>::run(C, Fs, X, rely, relz, row0, tw, zbuf, slot, batch, nzc);
    }
  }
};

template <int N, int ELL>
__global__ void __launch_bounds__(KZ_THREADS)
k_yz_rows(const float* __restrict__ mesh, int ix0, const float* __restrict__ relx, const float* __restrict__ rely,
          const float* __restrict__ relz, const float2* __restrict__ tw_g, float2* __restrict__ zbuf, int nzc,
          int batch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* C = tw + N;
  float* Fs = reinterpret_cast<float*>(C + KZ_ROWS * (N + 1));
  const int slot = blockIdx.y;
  const int ix = ix0 + slot;
  const int row0 = blockIdx.x * KZ_ROWS;
  for (int k = threadIdx.x; k < N; k += blockDim.x) tw[k] = tw_g[k];
  const float* src = mesh + ((size_t)ix * N + row0) * N;
  for (int k = threadIdx.x; k < KZ_ROWS * N / 4; k += blockDim.x)
    reinterpret_cast<float4*>(Fs)[k] = reinterpret_cast<const float4*>(src)[k];
  __syncthreads();
  PairLoop<N, ELL, 0>::run(C, Fs, relx[ix], rely, relz, row0, tw, zbuf, slot, batch, nzc);
}

template <int N, int ELL>
__global__ void __launch_bounds__(KY_THREADS)
k_yz_cols(const float2* __restrict__ zbuf, int ix0, int nzc, int batch, int kc, const int* __restrict__ col_off,
          const float2* __restrict__ tw_g, float2* __restrict__ gout, int mesh_j, int np) {
  using T = GroupTable<ELL>;
  constexpr int NB = T::NB, NG = T::NG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* S = tw + N;
  const int slot = blockIdx.y;
  const int ix = ix0 + slot;
  const int kz0 = blockIdx.x * kc;
  for (int k = threadIdx.x; k < N; k += blockDim.x) tw[k] = tw_g[k];
  const int nl = NB * kc;
  for (int e = threadIdx.x; e < nl * N; e += blockDim.x) {
    const int line = e / N, iy = e - (e / N) * N;
    const int f = line / kc, c = line - f * kc;
    const int kz = kz0 + c;
    S[line * (N + 1) + iy] =
        kz < nzc ? zbuf[(((size_t)f * batch + slot) * nzc + kz) * N + iy] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_smem<N, false>(S, 1, N + 1, nl, tw);
  for (int c = 0; c < kc; ++c) {
    const int kz = kz0 + c;
    if (kz >= nzc) break;
    const int p0 = col_off[kz];
    const int cnt = col_off[kz + 1] - p0;
    const int kymax = (cnt - 1) / 2;
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
      const int ky = q - kymax;
      const int iyk = ky < 0 ? ky + N : ky;
      float2 psi[NB];
#pragma unroll
      for (int f = 0; f < NB; ++f) psi[f] = S[(f * kc + c) * (N + 1) + iyk];
      float2 g[NG];
      T::combine(psi, (float)ky, (float)kz, g);
#pragma unroll
      for (int gi = 0; gi < NG; ++gi) gout[(((size_t)mesh_j * NG + gi) * N + ix) * np + p0 + q] = g[gi];
    }
  }
}

// Segmented (by key) inclusive sum within a warp; returns true on the last lane of
// each run of equal keys, which then holds the run total in v.
__device__ __forceinline__ bool warp_segment_sum(float& v, int key) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int kprev = __shfl_up_sync(full, key, 1);
  const int knext = __shfl_down_sync(full, key, 1);
  const bool head = lane == 0 || kprev != key;
  const bool tail = lane == 31 || knext != key;
  const unsigned heads = __ballot_sync(full, head);
  const unsigned mask = heads & ((lane == 31) ? full : ((2u << lane) - 1u));
  const int start = 31 - __clz(mask);
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float vo = __shfl_up_sync(full, v, o);
    if (lane - o >= start) v += vo;
  }
  return tail;
}

// Pencils per CTA of k_x_combine.
__host__ __device__ constexpr int k3_pencils(int n) { return n <= 32 ? 32 : (n >= 1024 ? 4 : 8); }

template <int N, int ELL, int M>
struct XCombine {
  static constexpr int P = k3_pencils(N);
  static constexpr int E = fft_elems(N);
  static constexpr int THREADS = P * (N / E);
  static constexpr int NW = THREADS / 32;
  static constexpr int ITEMS = P * N / 32;           // runs of 32 consecutive (pencil, k_x) modes
  static constexpr int K = ITEMS / NW;               // modes per thread
  static_assert(THREADS % 32 == 0, "threads");
  static_assert(ITEMS % NW == 0, "items");
};

template <int N, int ELL, int M>
__global__ void __launch_bounds__(XCombine<N, ELL, M>::THREADS)
k_x_combine(const float2* __restrict__ gin, int np, const short2* __restrict__ pencil, const float2* __restrict__ tw_g,
            const float* __restrict__ invw_g, const float2* __restrict__ phase_g, const short* __restrict__ lut,
            int n2_hi, double* __restrict__ acc, int nbins) {
  using XC = XCombine<N, ELL, M>;
  constexpr int P = XC::P, K = XC::K, NW = XC::NW, PP = P + 1;
  constexpr int NG = GroupTable<ELL>::NG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sbin = reinterpret_cast<double*>(smem_raw);                 // [3][nbins]
  float2* tw = reinterpret_cast<float2*>(sbin + 3 * nbins);          // [N]
  float2* phs = tw + N;                                              // [N]
  float* invw = reinterpret_cast<float*>(phs + N);                   // [N]
  short2* spen = reinterpret_cast<short2*>(invw + N);                // [P]
  float2* T = reinterpret_cast<float2*>(spen + P + (P & 1));         // [N][P + 1]
  for (int k = threadIdx.x; k < 3 * nbins; k += blockDim.x) sbin[k] = 0.0;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    tw[k] = tw_g[k];
    phs[k] = phase_g[k];
    invw[k] = invw_g[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int npb = (np + P - 1) / P;
  for (int pb = blockIdx.x; pb < npb; pb += gridDim.x) {
    __syncthreads();
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
      const int pi = pb * P + k;
      spen[k] = pi < np ? pencil[pi] : make_short2(0, -1);
    }
    __syncthreads();
    float2 a0[K], ga[K];
    // A single pass over (mesh, group) tiles; groups are visited in order A_0, then
    // the k_x powers of A_2, then those of A_4.
    for (int gi = 0; gi < NG; ++gi) {
      for (int mj = 0; mj < M; ++mj) {
        const float2* src = gin + ((size_t)(mj * NG + gi) * N) * np + (size_t)pb * P;
        for (int e = threadIdx.x; e < N * P; e += blockDim.x) {
          const int ix = e / P, p = e - (e / P) * P;
          T[ix * PP + p] = (pb * P + p < np) ? src[(size_t)ix * np + p] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        fft_smem<N, true>(T, PP, 1, P, tw);
        const int pw = (gi == 0) ? 0 : (gi <= 3 ? gi - 1 : gi - 4);  // power of k_x
#pragma unroll
        for (int q = 0; q < K; ++q) {
          const int flat = (warp + NW * q) * 32 + lane;
          const int p = flat / N, kx = flat - (flat / N) * N;
          const short2 pc = spen[p];
          const int ky = pc.x, kz = pc.y;
          const int mx = kx <= N / 2 ? kx : kx - N;
          const int iyk = ky < 0 ? ky + N : ky;
          float cf = invw[kx] * invw[iyk] * invw[kz < 0 ? 0 : kz] * (M == 2 ? 0.5f : 1.f);
          float2 X = T[kx * PP + p];
          if (M == 2 && mj == 1) {
            const float2 ph = cmul(cmul(phs[kx], phs[iyk]), phs[kz < 0 ? 0 : kz]);
            X = cmul(X, ph);
          }
          float kp = cf;
          for (int t = 0; t < pw; ++t) kp *= (float)mx;
          if (gi == 0) {
            if (mj == 0) a0[q] = make_float2(kp * X.x, kp * X.y);
            else { a0[q].x = fmaf(kp, X.x, a0[q].x); a0[q].y = fmaf(kp, X.y, a0[q].y); }
          } else {
            const bool first = (gi == 1 || gi == 4) && mj == 0;
            if (first) ga[q] = make_float2(kp * X.x, kp * X.y);
            else { ga[q].x = fmaf(kp, X.x, ga[q].x); ga[q].y = fmaf(kp, X.y, ga[q].y); }
          }
        }
        __syncthreads();
      }
      // After the last tile of A_0, of A_2 (gi == 3) or of A_4 (gi == 8): shell sums.
      const int slot = (gi == 0) ? 0 : (gi == 3 ? 1 : (gi == 8 ? 2 : -1));
      if (slot >= 0) {
#pragma unroll
        for (int q = 0; q < K; ++q) {
          const int flat = (warp + NW * q) * 32 + lane;
          const int p = flat / N, kx = flat - (flat / N) * N;
          const short2 pc = spen[p];
          const int ky = pc.x, kz = pc.y;
          const int mx = kx <= N / 2 ? kx : kx - N;
          const int n2 = mx * mx + ky * ky + kz * kz;
          int bin = -1;
          if (kz >= 0 && n2 < n2_hi) bin = lut[n2];
          const float wgt = (bin >= 0) ? (kz == 0 ? 1.f : 2.f) : 0.f;
          float v;
          if (slot == 0) {
            v = wgt * (a0[q].x * a0[q].x + a0[q].y * a0[q].y);
          } else {
            const float inv = n2 > 0 ? 1.f / (float)n2 : 0.f;
            const float invn = slot == 1 ? inv : inv * inv;
            v = wgt * invn * (a0[q].x * ga[q].x + a0[q].y * ga[q].y);
          }
          if (warp_segment_sum(v, bin) && bin >= 0) atomicAdd(&sbin[slot * nbins + bin], (double)v);
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 3 * nbins; k += blockDim.x)
    if (sbin[k] != 0.0) atomicAdd(&acc[k], sbin[k]);
}

template <int N, int ELL, int M>
size_t x_combine_smem(int nbins) {
  constexpr int P = k3_pencils(N);
  size_t b = sizeof(double) * 3 * nbins + sizeof(float2) * 2 * N + sizeof(float) * N + sizeof(short2) * (P + (P & 1));
  b = (b + 15) & ~size_t(15);
  return b + sizeof(float2) * N * (P + 1);
}

}  // namespace ys
