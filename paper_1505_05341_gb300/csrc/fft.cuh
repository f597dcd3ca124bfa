// Shared-memory complex FFTs for the mesh transforms (forward, e^{-2 pi i j k / N}).
//
// The method (Sec. 3) places no condition on the FFT algorithm; this one is a
// Stockham autosort decimation-in-time transform with the result in natural order.
// N is 2^a (radix-8 stages, then one radix-4 or radix-2) or 3 * 2^a (radix-4 stages,
// an optional radix-2, then radix-3).  Each thread holds E = 8 (or 12) elements per
// line and does E / R butterflies per stage; the data go through shared memory
// between stages.  Twiddles come from a stage-major table (fft_tw_offset) computed
// in FP64 on the host and rounded to float.
#pragma once
#include <cuda_runtime.h>

namespace ys {

__host__ __device__ constexpr bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Elements per thread.  Walked by consecutive threads (y,z stage), a line fits one
// warp up to N = 512 (768); its TPL = N / E threads synchronise among themselves only
// (line_group_sync).  Interleaved lines (x stage) use 8 or 12 elements.
__host__ __device__ constexpr int fft_elems(int n) {
  return is_pow2(n) ? 8 : 12;
}
__host__ __device__ constexpr int fft_elems_lf(int n) { return is_pow2(n) ? 8 : 12; }

// Barrier over the TPL consecutive threads that own one line: the warp when the
// line fits in it, else a named barrier (ids 1..15) shared by those threads only.
template <int TPL>
__device__ __forceinline__ void line_group_sync() {
  if constexpr (TPL <= 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / TPL)), "r"(TPL) : "memory");
  }
}

// Number of stages and the radix of stage s (see header comment).
__host__ __device__ constexpr int fft_nstages(int n) {
  if (is_pow2(n)) {
    int s = 0, m = n;
    while (m >= 8) { m /= 8; ++s; }
    return s + (m > 1 ? 1 : 0);
  }
  int s = 0, m = n / 3;
  while (m % 4 == 0) { m /= 4; ++s; }
  return s + (m == 2 ? 1 : 0) + 1;
}

__host__ __device__ constexpr int fft_radix(int n, int stage) {
  if (is_pow2(n)) {
    int m = n, s = 0;
    while (m >= 8) { if (s == stage) return 8; m /= 8; ++s; }
    return m;
  }
  int m = n / 3, s = 0;
  while (m % 4 == 0) { if (s == stage) return 4; m /= 4; ++s; }
  if (m == 2) { if (s == stage) return 2; ++s; }
  return 3;
}

__host__ __device__ constexpr int fft_ns_before(int n, int stage) {
  int ns = 1;
  for (int s = 0; s < stage; ++s) ns *= fft_radix(n, s);
  return ns;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// Complex sums and differences use the packed two-lane float instructions of
// sm_100-class GPUs (one instruction for both components).  a - b is formed as
// fma(b, -1, a), whose product is exact, so it rounds exactly as a - b does.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 cswap(float2 a) { return make_float2(a.y, a.x); }
// a + (-i) t and a - (-i) t
__device__ __forceinline__ float2 add_mi(float2 a, float2 t) { return __ffma2_rn(cswap(t), make_float2(1.f, -1.f), a); }
__device__ __forceinline__ float2 sub_mi(float2 a, float2 t) { return __ffma2_rn(cswap(t), make_float2(-1.f, 1.f), a); }
// a + s t for a real s given as (s, s)
__device__ __forceinline__ float2 cfma(float2 t, float2 s, float2 a) { return __ffma2_rn(t, s, a); }

template <int R> struct Dft;

template <> struct Dft<2> {
  __device__ static __forceinline__ void run(float2* v) {
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <> struct Dft<3> {
  __device__ static __forceinline__ void run(float2* v) {
    // w = e^{-2 pi i / 3} = -1/2 - i sqrt(3)/2
    const float s3 = 0.866025403784438647f;
    const float2 a = v[0], b = v[1], c = v[2];
    const float2 t1 = cadd(b, c);
    const float2 t2 = cfma(t1, make_float2(-0.5f, -0.5f), a);
    const float2 d = csub(b, c);
    // t2 +/- (-i sqrt3/2) d
    v[0] = cadd(a, t1);
    v[1] = cfma(cswap(d), make_float2(s3, -s3), t2);
    v[2] = cfma(cswap(d), make_float2(-s3, s3), t2);
  }
};

template <> struct Dft<4> {
  __device__ static __forceinline__ void run(float2* v) {
    const float2 a = v[0], b = v[1], c = v[2], d = v[3];
    const float2 s0 = cadd(a, c), s1 = csub(a, c);
    const float2 s2 = cadd(b, d), t = csub(b, d);
    v[0] = cadd(s0, s2);
    v[2] = csub(s0, s2);
    v[1] = add_mi(s1, t);
    v[3] = sub_mi(s1, t);
  }
};

template <> struct Dft<8> {
  __device__ static __forceinline__ void run(float2* v) {
    // even / odd split into two DFT-4s, then w8^k = e^{-i pi k / 4}.
    const float h = 0.707106781186547524f;
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    Dft<4>::run(e);
    Dft<4>::run(o);
    // w8 o1 = h u1 with u1 = (o1.x + o1.y, o1.y - o1.x); w8^3 o3 = -h u3 with
    // u3 = (o3.x - o3.y, o3.y + o3.x); w8^2 o2 = -i o2.
    const float2 u1 = add_mi(o[1], o[1]);
    const float2 u3 = sub_mi(o[3], o[3]);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cfma(u1, make_float2(h, h), e[1]);
    v[5] = cfma(u1, make_float2(-h, -h), e[1]);
    v[2] = add_mi(e[2], o[2]);
    v[6] = sub_mi(e[2], o[2]);
    v[3] = cfma(u3, make_float2(-h, -h), e[3]);
    v[7] = cfma(u3, make_float2(h, h), e[3]);
  }
};

// Element offset inside a line: with PAD, one complex of padding follows every 16
// elements.  A float2 access is served per half-warp over 16 bank pairs, so 16
// consecutive elements that start on a multiple of 16 stay on 16 distinct pairs,
// while the strided Stockham stores (element R j + r, R = 8 or 4) are spread over the
// pairs by the pad.
template <bool PAD>
__host__ __device__ constexpr int fft_pos(int i) { return PAD ? i + (i >> 4) : i; }

// Line length in complex elements for a padded / unpadded layout.  Padded lines are
// 1 mod 16 (lines read at one element by 16 row lanes land on 16 pairs), or 2 mod 16
// when ROWS_ARE_PAIRS (8 rows x 2 elements per half-warp, the split of the y,z
// stage's row items from 512^3 up); unpadded ones are odd.
template <int N, bool PAD, bool ROWS_ARE_PAIRS = false>
__host__ __device__ constexpr int fft_line_len() {
  if (!PAD) return N + 1;
  const int base = N + N / 16;
  const int want = ROWS_ARE_PAIRS ? 2 : 1;
  return base + ((want - base % 16) + 16) % 16;
}

// Twiddles are stored stage by stage: for stage s >= 1 (N_s = fft_ns_before(N, s)
// elements already combined, radix R_s), entry k (R_s - 1) + r - 1 of the stage's
// block is exp(-2 pi i r k / (N_s R_s)), k < N_s, 1 <= r < R_s.  A butterfly then
// reads its R_s - 1 twiddles from one base address.  The blocks fill N - R_0 < N
// entries in all.
__host__ __device__ constexpr int fft_tw_offset(int n, int stage) {
  int off = 0;
  for (int s = 1; s < stage; ++s) off += fft_ns_before(n, s) * (fft_radix(n, s) - 1);
  return off;
}

// One Stockham stage over `nl` lines of length N stored in shared memory at
// buf[line * ls + elem * es].  LF: consecutive threads take consecutive lines (for
// layouts whose lines interleave); otherwise consecutive threads walk one line.
// NL > 0: the number of lines is a compile-time constant (passes unrolled, separated
// by a line-group barrier so that no pass's addresses are hoisted into another);
// NL == 0: nl lines at run time.
//
// Padded lines walked by consecutive threads (the y,z stage) take a fast path: element
// i sits at i + i/16, and (a + 16 m)/16 = a/16 + m, so when the threads per line and
// the input stride are multiples of 16 every load is one per-thread base address plus
// a compile-time offset.  The stores go to outb + r N_s with outb = k (mod N_s R): for
// N_s a multiple of 16 the same holds, and for N_s dividing 16 (with k < N_s and N_s R
// a multiple of 16) element outb + r N_s sits at pos(outb) + r N_s + (r N_s)/16.
template <int N, int S, bool LF, bool PAD, int NL = 0>
__device__ __forceinline__ void fft_stage(float2* buf, int es, int ls, int nl_rt, const float2* tw) {
  constexpr int R = fft_radix(N, S);
  constexpr int E = LF ? fft_elems_lf(N) : fft_elems(N);
  constexpr int TPL = N / E;        // threads per line
  constexpr int NB = E / R;         // butterflies per thread
  constexpr int NS = fft_ns_before(N, S);
  constexpr int STRIDE = N / R;
  constexpr bool FAST_LD = !LF && PAD && TPL % 16 == 0 && STRIDE % 16 == 0;
  constexpr bool FAST_ST = !LF && PAD && (NS % 16 == 0 || (16 % NS == 0 && (NS * R) % 16 == 0));
  const float2* tws = tw + fft_tw_offset(N, S);
  // Lines walked by consecutive threads only need their own threads synchronised.
  const int tid = threadIdx.x;
  const int lpp = blockDim.x / TPL;  // lines per pass
  const bool in_pass = tid < lpp * TPL;
  const int lane_line = LF ? tid % lpp : tid / TPL;
  const int tl = LF ? tid / lpp : tid % TPL;
  const int nl = NL > 0 ? NL : nl_rt;
#pragma unroll 1
  for (int base_line = 0; base_line < nl; base_line += lpp) {
    const int line = base_line + lane_line;
    const bool ok = in_pass && line < nl;
    float2 v[E];
    if (ok) {
      const float2* lp = buf + line * ls;
      if constexpr (FAST_LD) {
        const float2* src = lp + (tl + (tl >> 4));
#pragma unroll
        for (int q = 0; q < NB; ++q)
#pragma unroll
          for (int r = 0; r < R; ++r) v[q * R + r] = src[(q * TPL + r * STRIDE) / 16 * 17];
      } else {
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          const int j = tl + q * TPL;
#pragma unroll
          for (int r = 0; r < R; ++r) v[q * R + r] = lp[fft_pos<PAD>(j + r * STRIDE) * es];
        }
      }
    }
    if constexpr (LF) __syncthreads(); else line_group_sync<TPL>();
    if (ok) {
      float2* lp = buf + line * ls;
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        const int j = tl + q * TPL;
        const int k = j % NS;
        if (NS > 1) {
          const float2* tk = tws + k * (R - 1);
#pragma unroll
          for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], tk[r - 1]);
        }
        Dft<R>::run(&v[q * R]);
        const int outb = (j / NS) * NS * R + k;
        if constexpr (FAST_ST) {
          float2* dst = lp + (outb + (outb >> 4));
#pragma unroll
          for (int r = 0; r < R; ++r) dst[r * NS + (r * NS) / 16] = v[q * R + r];
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) lp[fft_pos<PAD>(outb + r * NS) * es] = v[q * R + r];
        }
      }
    }
    if constexpr (LF) __syncthreads(); else line_group_sync<TPL>();
  }
}

// Padded buffers of interleaved lines (x stage: element x of line p at x P + p):
// PADP > 0 inserts PADP elements after every 8 PADP, so that the stores of a radix-8
// first stage, 8 P apart across a warp, land on distinct bank pairs.
template <int PADP>
__host__ __device__ constexpr int lf_pad(int i) {
  return PADP > 0 ? i + (i / (8 * PADP)) * PADP : i;
}

// Out-of-place stage: reads the lines from src and writes them to dst (no barrier
// inside; the caller synchronises before dst is read).  With two buffers a stage
// needs one barrier instead of the two an in-place stage needs.  PIN / POUT: the
// padding (lf_pad) of src / dst.
template <int N, int S, bool LF, int PIN = 0, int POUT = 0>
__device__ __forceinline__ void fft_stage_oop(const float2* src, float2* dst, int es, int ls, int nl,
                                              const float2* tw) {
  constexpr int R = fft_radix(N, S);
  constexpr int E = LF ? fft_elems_lf(N) : fft_elems(N);
  constexpr int TPL = N / E;
  constexpr int NB = E / R;
  constexpr int NS = fft_ns_before(N, S);
  constexpr int STRIDE = N / R;
  const float2* tws = tw + fft_tw_offset(N, S);
  const int tid = threadIdx.x;
  const int lpp = blockDim.x / TPL;
  const bool in_pass = tid < lpp * TPL;
  const int lane_line = LF ? tid % lpp : tid / TPL;
  const int tl = LF ? tid / lpp : tid % TPL;
#pragma unroll 1
  for (int base_line = 0; base_line < nl; base_line += lpp) {
    const int line = base_line + lane_line;
    if (!in_pass || line >= nl) continue;
    const int lo = line * ls;
    float2 v[E];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int j = tl + q * TPL;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = src[lf_pad<PIN>(lo + (j + r * STRIDE) * es)];
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int j = tl + q * TPL;
      const int k = j % NS;
      if (NS > 1) {
        const float2* tk = tws + k * (R - 1);
#pragma unroll
        for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], tk[r - 1]);
      }
      Dft<R>::run(&v[q * R]);
      const int outb = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[lf_pad<POUT>(lo + (outb + r * NS) * es)] = v[q * R + r];
    }
  }
}

// Stages [S, END) alternating between buffers a and b (CTA-wide barrier after each);
// the result sits in a when END - S is even, else in b.  PA / PB: their padding.
template <int N, int S, int END, int PA = 0, int PB = 0, bool Done = (S >= END)>
struct FftPingPong {
  __device__ static __forceinline__ void run(float2* a, float2* b, int es, int ls, int nl, const float2* tw) {
    fft_stage_oop<N, S, true, PA, PB>(a, b, es, ls, nl, tw);
    __syncthreads();
    FftPingPong<N, S + 1, END, PB, PA>::run(b, a, es, ls, nl, tw);
  }
};
template <int N, int S, int END, int PA, int PB>
struct FftPingPong<N, S, END, PA, PB, true> {
  __device__ static __forceinline__ void run(float2*, float2*, int, int, int, const float2*) {}
};

// Terminate the recursion at S == number of stages.
template <int N, int S, bool LF, bool PAD = false, int NL = 0, bool Done = (S >= fft_nstages(N))>
struct FftRun {
  __device__ static __forceinline__ void run(float2* buf, int es, int ls, int nl, const float2* tw) {
    fft_stage<N, S, LF, PAD, NL>(buf, es, ls, nl, tw);
    FftRun<N, S + 1, LF, PAD, NL>::run(buf, es, ls, nl, tw);
  }
};
template <int N, int S, bool LF, bool PAD, int NL>
struct FftRun<N, S, LF, PAD, NL, true> {
  __device__ static __forceinline__ void run(float2*, int, int, int, const float2*) {}
};

// Last stage into registers: stages 0 .. S-2 must already have run on the lines.
// Each thread loads its butterfly inputs from line `line` of buf (element i at
// line + i es, padded by lf_pad<PADL>), applies twiddles and the DFT, and keeps the
// outputs: v[q * R + r] is element (tl + q * TPL) + r * (N / R).
template <int N, bool LF, bool PAD, int PADL = 0>
__device__ __forceinline__ void fft_last_stage_regs(const float2* buf, int line, int es, int tl, const float2* tw,
                                                    float2 (&v)[LF ? fft_elems_lf(N) : fft_elems(N)]) {
  constexpr int S = fft_nstages(N) - 1;
  constexpr int R = fft_radix(N, S);
  constexpr int E = LF ? fft_elems_lf(N) : fft_elems(N);
  constexpr int TPL = N / E;
  constexpr int NB = E / R;
  constexpr int NS = fft_ns_before(N, S);
  constexpr int STRIDE = N / R;
  const float2* tws = tw + fft_tw_offset(N, S);
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int j = tl + q * TPL;
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = buf[lf_pad<PADL>(line + fft_pos<PAD>(j + r * STRIDE) * es)];
  }
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    const int j = tl + q * TPL;
    const int k = j % NS;
    if (NS > 1) {
      const float2* tk = tws + k * (R - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], tk[r - 1]);
    }
    Dft<R>::run(&v[q * R]);
  }
}

// First stage from registers: the caller holds, for its butterflies q < E/R0, the
// inputs v[q * R0 + r] = x[fft_in_index<N>(tl, q, r)] of one line; this does the
// stage-0 butterflies (no twiddles: N_s = 1) and stores the results to the line lp.
// The remaining stages run with FftRun<N, 1, LF> after a line-group barrier.
template <int N>
__host__ __device__ constexpr int fft_in_index(int tl, int q, int r) {
  return tl + q * (N / fft_elems(N)) + r * (N / fft_radix(N, 0));
}

template <int N, bool PAD>
__device__ __forceinline__ void fft_stage0_regs(float2 (&v)[fft_elems(N)], float2* lp, int es, int tl) {
  constexpr int R = fft_radix(N, 0);
  constexpr int E = fft_elems(N);
  constexpr int TPL = N / E;
#pragma unroll
  for (int q = 0; q < E / R; ++q) {
    Dft<R>::run(&v[q * R]);
    const int j = tl + q * TPL;
    if constexpr (PAD && 16 % R == 0) {
      float2* dst = lp + fft_pos<true>(j * R) * es;  // element R j + r sits r after R j (R | 16)
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * es] = v[q * R + r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) lp[fft_pos<PAD>(j * R + r) * es] = v[q * R + r];
    }
  }
}

}  // namespace ys
