// The two direct-sum estimators of Sec. 4, "sum-gal" and "sum-grid", on the GPU.
//
// Both evaluate Eq. (4) with A_n(k) = sum_p s_p w_p (k_hat . r_hat_p)^n e^{-i k.x_p} at
// every half-grid mode k = k_F m of the binning, for n = 0, 2, 4 (and 6), then the
// shell means of Eqs. (6)-(8):
//   sum-gal   the points are the galaxies (s = +1) and randoms (s = -alpha), r_p the
//             point's own line of sight: no mesh, no window, no aliasing, and any
//             k lattice (k_F m with |m| below n_mesh / 2 of the configuration, which
//             need not be an FFT size);
//   sum-grid  the points are the nodes of a plan's assigned mesh(es), weight F,
//             r = node - observer as in the FFT path: its exact DFT, which the FFT
//             path reproduces mode by mode.
// One more complex sum per mode, with the top hat Theta(|mu| <= 1/2) in place of the
// Legendre weight, gives the wedges by their definition (Sec. 5, Eqs. 14-15).
//
// Layout: one thread per mode, with the mode's complex sums in registers; points
// stream through shared memory in chunks that every thread reads as broadcasts.
// Positions are 32-bit fixed-point fractions of the box, u = (x - box_min) / L, so
// the phase k.x = 2 pi m.u is taken mod one turn exactly by integer multiply-adds;
// only the final angle in [-pi, pi) is rounded.  Each thread's sums are compensated
// float (TwoSum per add); CTAs that split the points add their sums into FP64
// per-mode accumulators, and a second kernel forms the shell sums in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "ys_internal.h"

namespace ys {
namespace {

constexpr int SG_THREADS = 256;
constexpr int SG_CHUNK = 256;  // points per shared-memory chunk

// Components of the per-mode sums: A_0, A_2, A_4, A_6 and the top-hat sum B_perp.
enum { C_A0 = 0, C_A2 = 1, C_A4 = 2, C_A6 = 3, C_BP = 4, C_COUNT = 5 };

struct SgPoint {
  uint32_t u[3];  // position as a fraction of the box, 2^-32 units
  float sw;       // signed weight
  float rh[3];    // r_hat (0 at r = 0)
  float pad;
};

struct SgMode {
  short m[3];     // integer frequency
  short bin;      // shell
  float khat[3];
  float w;        // Hermitian weight (1 or 2)
};

__device__ __forceinline__ float two_sum_err(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return (a - (s - bb)) + (b - bb);
}

// s += v with its exact rounding error added to c.
__device__ __forceinline__ void add_comp(float& s, float& c, float v) {
  const float t = s + v;
  c += two_sum_err(s, v);
  s = t;
}

// FP64 catalogue sums of Eqs. (1) and (3) (the same slots as the assignment's).
__global__ void k_sg_sums(const float* __restrict__ w, const float* __restrict__ nbar, int64_t n, int is_ran,
                          double* __restrict__ sums) {
  double s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = w ? (double)w[i] : 1.0;
    s1 += v;
    s2 += v * v;
    if (is_ran && nbar) s3 += v * v * (double)nbar[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s3 += __shfl_xor_sync(0xffffffffu, s3, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (is_ran) {
      atomicAdd(&sums[SUM_WR], s1);
      atomicAdd(&sums[SUM_WR2], s2);
      atomicAdd(&sums[SUM_WR2N], s3);
    } else {
      atomicAdd(&sums[SUM_WG], s1);
      atomicAdd(&sums[SUM_WG2], s2);
    }
  }
}

__device__ __forceinline__ uint32_t to_fixed(double u) {
  u -= floor(u);  // one period of the box (the sums are periodic in x with period L)
  return (uint32_t)(uint64_t)(u * 4294967296.0);
}

__device__ __forceinline__ void unit3(double x, double y, double z, float (&o)[3]) {
  const double r = sqrt(x * x + y * y + z * z);
  const double inv = r > 0.0 ? 1.0 / r : 0.0;
  o[0] = (float)(x * inv);
  o[1] = (float)(y * inv);
  o[2] = (float)(z * inv);
}

// Catalogue particles as points: galaxies +w, randoms -alpha w.
__global__ void k_sg_points_cat(const float* __restrict__ x, const float* __restrict__ y,
                                const float* __restrict__ z, const float* __restrict__ w, int64_t n, int is_ran,
                                const double* __restrict__ sums, double alpha_cfg, double bx, double by, double bz,
                                double inv_len, double ox, double oy, double oz, SgPoint* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double sgn = 1.0;
  if (is_ran) sgn = -(alpha_cfg >= 0.0 ? alpha_cfg : sums[SUM_WG] / sums[SUM_WR]);
  const double px = x[i], py = y[i], pz = z[i];
  SgPoint q;
  q.u[0] = to_fixed((px - bx) * inv_len);
  q.u[1] = to_fixed((py - by) * inv_len);
  q.u[2] = to_fixed((pz - bz) * inv_len);
  q.sw = (float)(sgn * (w ? (double)w[i] : 1.0));
  unit3(px - ox, py - oy, pz - oz, q.rh);
  q.pad = 0.f;
  out[i] = q;
}

// Mesh nodes [first, first + count) of mesh j with F != 0 as points (compacted with a
// counter).  Node i of mesh j sits at box_min + (i + j/2) H; scale multiplies F (1/2
// for each of two interlaced meshes).
__global__ void k_sg_points_mesh(const float* __restrict__ mesh, int n, int j, int64_t first, int64_t count_nodes,
                                 double rel_x0, double rel_y0, double rel_z0, double H, float scale,
                                 unsigned* __restrict__ count, SgPoint* __restrict__ out) {
  const int64_t idx = first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= first + count_nodes) return;
  const float f = mesh[idx];
  if (f == 0.f) return;
  const int iz = (int)(idx % n), iy = (int)((idx / n) % n), ix = (int)(idx / ((int64_t)n * n));
  const double s = 0.5 * j;
  SgPoint q;
  const double inv_n = 1.0 / n;
  q.u[0] = to_fixed((ix + s) * inv_n);
  q.u[1] = to_fixed((iy + s) * inv_n);
  q.u[2] = to_fixed((iz + s) * inv_n);
  q.sw = f * scale;
  unit3(rel_x0 + (ix + s) * H, rel_y0 + (iy + s) * H, rel_z0 + (iz + s) * H, q.rh);
  q.pad = 0.f;
  out[atomicAdd(count, 1u)] = q;
}

// Per-mode sums over the points [p_lo, p_hi) of this CTA's split; FP64 atomics into
// acc[C_COUNT][nmodes] (interleaved re, im).
template <int ELL, bool WEDGE>
__global__ void __launch_bounds__(SG_THREADS) k_sg_modes(const SgMode* __restrict__ modes, int nmodes,
                                                          const SgPoint* __restrict__ pts,
                                                          const unsigned* __restrict__ npts_dev, int64_t npts_host,
                                                          int splits, double* __restrict__ acc) {
  __shared__ SgPoint s_pts[SG_CHUNK];
  const int mi = blockIdx.x * SG_THREADS + threadIdx.x;
  const bool active = mi < nmodes;
  const int64_t npts = npts_dev ? (int64_t)*npts_dev : npts_host;
  const int64_t per = (npts + splits - 1) / splits;
  const int64_t p_lo = std::min<int64_t>(npts, per * blockIdx.y), p_hi = std::min<int64_t>(npts, p_lo + per);
  int mx = 0, my = 0, mz = 0;
  float kx = 0.f, ky = 0.f, kz = 0.f;
  if (active) {
    const SgMode md = modes[mi];
    mx = md.m[0];
    my = md.m[1];
    mz = md.m[2];
    kx = md.khat[0];
    ky = md.khat[1];
    kz = md.khat[2];
  }
  constexpr int NC = (ELL >= 6 ? 4 : ELL / 2 + 1) + (WEDGE ? 1 : 0);
  float sre[NC], sim[NC], cre[NC], cim[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) sre[c] = sim[c] = cre[c] = cim[c] = 0.f;
  for (int64_t base = p_lo; base < p_hi; base += SG_CHUNK) {
    const int cnt = (int)std::min<int64_t>(SG_CHUNK, p_hi - base);
    __syncthreads();
    if (threadIdx.x < cnt) s_pts[threadIdx.x] = pts[base + threadIdx.x];
    __syncthreads();
    if (!active) continue;
    for (int j = 0; j < cnt; ++j) {
      const SgPoint q = s_pts[j];
      // one turn = 2^32: the phase m.u mod 1 is exact in wrapping integer arithmetic
      const uint32_t turn = (uint32_t)mx * q.u[0] + (uint32_t)my * q.u[1] + (uint32_t)mz * q.u[2];
      float sn, cs;
      sincospif((float)(int32_t)turn * 4.656612873077393e-10f, &sn, &cs);  // angle / pi in [-1, 1)
      const float tre = q.sw * cs, tim = -q.sw * sn;                        // s w e^{-i k.x}
      add_comp(sre[0], cre[0], tre);
      add_comp(sim[0], cim[0], tim);
      if constexpr (ELL >= 2 || WEDGE) {
        const float mu = fmaf(kx, q.rh[0], fmaf(ky, q.rh[1], kz * q.rh[2]));
        const float mu2 = mu * mu;
        float f = mu2;
#pragma unroll
        for (int c = 1; c <= (ELL >= 6 ? 3 : ELL / 2); ++c) {
          add_comp(sre[c], cre[c], f * tre);
          add_comp(sim[c], cim[c], f * tim);
          f *= mu2;
        }
        if constexpr (WEDGE) {
          const float t = fabsf(mu) <= 0.5f ? 1.f : 0.f;
          add_comp(sre[NC - 1], cre[NC - 1], t * tre);
          add_comp(sim[NC - 1], cim[NC - 1], t * tim);
        }
      }
    }
  }
  if (!active) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int comp = (WEDGE && c == NC - 1) ? C_BP : c;
    double* a = acc + ((size_t)comp * nmodes + mi) * 2;
    atomicAdd(a, (double)sre[c] + (double)cre[c]);
    atomicAdd(a + 1, (double)sim[c] + (double)cim[c]);
  }
}

// Shell sums in FP64: slot s = Re A_0 A_{2s}^* for s < nmain and, with wedge, slot 4 =
// Re A_0 B_perp^*, weighted; the window is divided out of every A (invw per axis, 1
// without it).
__global__ void k_sg_shells(const SgMode* __restrict__ modes, int nmodes, const double* __restrict__ acc,
                            const float* __restrict__ invw, int n, int nmain, int wedge, int nbins,
                            double* __restrict__ shell_acc) {
  const int mi = blockIdx.x * blockDim.x + threadIdx.x;
  if (mi >= nmodes) return;
  const SgMode md = modes[mi];
  double cw = 1.0;
  if (invw) {
    for (int a = 0; a < 3; ++a) {
      const int idx = md.m[a] < 0 ? md.m[a] + n : md.m[a];
      cw *= (double)invw[idx];
    }
  }
  const double* a0 = acc + (size_t)mi * 2;
  const double r0 = a0[0] * cw, i0 = a0[1] * cw;
  for (int s = 0; s < nmain + (wedge ? 1 : 0); ++s) {
    const int comp = s < nmain ? s : C_BP;
    const int slot = s < nmain ? s : 4;
    const double* as = acc + ((size_t)comp * nmodes + mi) * 2;
    const double v = md.w * (r0 * as[0] * cw + i0 * as[1] * cw);
    atomicAdd(&shell_acc[(size_t)slot * nbins + md.bin], v);
  }
}

// Result row (plan layout) and the wedges from the shell sums.
__global__ void k_sg_finalize(const double* __restrict__ sacc, const double* __restrict__ shell,
                              const double* __restrict__ sums, double alpha_cfg, int nbins, int ell, int wedges,
                              double* __restrict__ res, double* __restrict__ wout) {
  const double alpha = alpha_cfg >= 0.0 ? alpha_cfg : sums[SUM_WG] / sums[SUM_WR];
  const double I = alpha * sums[SUM_WR2N];
  const double S = sums[SUM_WG2] + alpha * alpha * sums[SUM_WR2];
  const double nan = __longlong_as_double(0x7ff8000000000000ULL);
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    const double nm = shell[b];
    double km = nan, p0 = nan, p2 = nan, p4 = nan, p6 = nan, pp = nan, pq = nan;
    if (nm > 0.0) {
      km = shell[nbins + b] / nm;
      const double m0 = sacc[b] / nm, m2 = sacc[nbins + b] / nm, m4 = sacc[2 * nbins + b] / nm;
      p0 = (m0 - S) / I;  // Eqs. (6)-(8)
      if (ell >= 2) p2 = 2.5 / I * (3.0 * m2 - m0);
      if (ell >= 4) p4 = 1.125 / I * (35.0 * m4 - 30.0 * m2 + 3.0 * m0);
      if (ell >= 6) p6 = 0.8125 / I * (231.0 * sacc[3 * nbins + b] / nm - 315.0 * m4 + 105.0 * m2 - 5.0 * m0);
      if (wedges) {  // Eqs. 14-15: the top hats normalised by 1 / (1/2), shot noise S/I
        const double mp = sacc[4 * nbins + b] / nm;
        pp = 2.0 / I * mp - S / I;
        pq = 2.0 / I * (m0 - mp) - S / I;
      }
    }
    res[b] = km;
    res[nbins + b] = nm;
    res[2 * nbins + b] = p0;
    res[3 * nbins + b] = p2;
    res[4 * nbins + b] = p4;
    if (ell >= 6) res[5 * nbins + 5 + b] = p6;
    if (wedges) {
      wout[b] = pp;
      wout[nbins + b] = pq;
    }
  }
  if (threadIdx.x == 0) {
    res[5 * nbins + 0] = alpha;
    res[5 * nbins + 1] = I;
    res[5 * nbins + 2] = S / I;
    res[5 * nbins + 3] = 0.0;
    res[5 * nbins + 4] = 0.0;
  }
}

struct ModeTable {
  std::vector<SgMode> modes;
  std::vector<double> shell;  // [2][nbins]: mode count, sum |k|
};

// Half-grid modes of an n^3 lattice (m_x, m_y in [-n/2, n/2), m_z in [0, n/2]; weight 2
// for 0 < m_z < n/2) with 0 < |k| < k_F n / 2 that fall in a shell.
ModeTable build_modes(const ys_config& c) {
  ModeTable t;
  const int n = c.n_mesh;
  const double kf = 2.0 * M_PI / c.box_len, knyq = kf * n / 2.0;
  const double kmax = std::min(knyq, c.k_min + c.dk * c.n_bins);
  const int mr = std::min(n / 2, (int)std::ceil(kmax / kf) + 1);
  t.shell.assign(2 * (size_t)c.n_bins, 0.0);
  for (int mx = -mr; mx <= mr; ++mx)
    for (int my = -mr; my <= mr; ++my)
      for (int mz = 0; mz <= mr; ++mz) {
        if (mx < -n / 2 || mx >= n / 2 || my < -n / 2 || my >= n / 2 || mz > n / 2) continue;
        const int n2 = mx * mx + my * my + mz * mz;
        if (n2 == 0) continue;
        const double km = kf * std::sqrt((double)n2);
        if (!(km < knyq)) continue;
        const double b = std::floor((km - c.k_min) / c.dk);
        if (!(b >= 0 && b < c.n_bins)) continue;
        SgMode md;
        md.m[0] = (short)mx;
        md.m[1] = (short)my;
        md.m[2] = (short)mz;
        md.bin = (short)b;
        const double inv = 1.0 / std::sqrt((double)n2);
        md.khat[0] = (float)(mx * inv);
        md.khat[1] = (float)(my * inv);
        md.khat[2] = (float)(mz * inv);
        md.w = (mz > 0 && mz < n / 2) ? 2.f : 1.f;
        t.modes.push_back(md);
        t.shell[(size_t)b] += md.w;
        t.shell[(size_t)c.n_bins + (size_t)b] += md.w * km;
      }
  return t;
}

// Device buffers of one direct-sum call, freed on every return path.
struct Scratch {
  std::vector<void*> ptrs;
  template <class T>
  cudaError_t get(T*& p, size_t count) {
    void* raw = nullptr;
    cudaError_t e = cudaMalloc(&raw, std::max<size_t>(1, count) * sizeof(T));
    if (!e) {
      ptrs.push_back(raw);
      p = static_cast<T*>(raw);
    }
    return e;
  }
  ~Scratch() {
    for (void* q : ptrs) cudaFree(q);
  }
};

ys_status fail(cudaError_t e) {
  g_last_cuda_error = cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? YS_ERR_OOM : YS_ERR_CUDA;
}

template <int ELL, bool WEDGE>
cudaError_t launch_modes(const SgMode* modes, int nmodes, const SgPoint* pts, const unsigned* npts_dev,
                         int64_t npts_host, double* acc, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e) return e;
  const int mblocks = (nmodes + SG_THREADS - 1) / SG_THREADS;
  // split the points so that the grid fills the GPU a few times over
  const int64_t want = (int64_t)sms * 8;
  int splits = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (want + mblocks - 1) / mblocks));
  const int64_t np_bound = npts_dev ? INT64_MAX : npts_host;
  splits = (int)std::max<int64_t>(1, std::min<int64_t>(splits, (np_bound + SG_CHUNK - 1) / SG_CHUNK));
  dim3 grid(mblocks, splits);
  k_sg_modes<ELL, WEDGE><<<grid, SG_THREADS, 0, st>>>(modes, nmodes, pts, npts_dev, npts_host, splits, acc);
  return cudaGetLastError();
}

cudaError_t run_modes(int ell, bool wedge, const SgMode* modes, int nmodes, const SgPoint* pts,
                      const unsigned* npts_dev, int64_t npts_host, double* acc, cudaStream_t st) {
  switch (ell * 2 + (wedge ? 1 : 0)) {
    case 0: return launch_modes<0, false>(modes, nmodes, pts, npts_dev, npts_host, acc, st);
    case 1: return launch_modes<0, true>(modes, nmodes, pts, npts_dev, npts_host, acc, st);
    case 4: return launch_modes<2, false>(modes, nmodes, pts, npts_dev, npts_host, acc, st);
    case 5: return launch_modes<2, true>(modes, nmodes, pts, npts_dev, npts_host, acc, st);
    case 8: return launch_modes<4, false>(modes, nmodes, pts, npts_dev, npts_host, acc, st);
    case 9: return launch_modes<4, true>(modes, nmodes, pts, npts_dev, npts_host, acc, st);
    case 12: return launch_modes<6, false>(modes, nmodes, pts, npts_dev, npts_host, acc, st);
    default: return launch_modes<6, true>(modes, nmodes, pts, npts_dev, npts_host, acc, st);
  }
}

// Shells, finalize and copies shared by both estimators.
ys_status finish(const ModeTable& mt, const SgMode* d_modes, const double* d_acc, const float* d_invw, int n,
                 const double* d_sums, double alpha_cfg, int nbins, int ell, bool wedge, double* d_out,
                 double* d_wedges, Scratch& sc, cudaStream_t st) {
  const int nmodes = (int)mt.modes.size();
  const int nmain = ell >= 6 ? 4 : ell / 2 + 1;
  const int slots_alloc = 5;
  double *d_sacc = nullptr, *d_shell = nullptr;
  cudaError_t e;
  if ((e = sc.get(d_sacc, (size_t)slots_alloc * nbins)) || (e = sc.get(d_shell, mt.shell.size()))) return fail(e);
  if ((e = cudaMemsetAsync(d_sacc, 0, sizeof(double) * slots_alloc * nbins, st))) return fail(e);
  if ((e = cudaMemcpyAsync(d_shell, mt.shell.data(), sizeof(double) * mt.shell.size(), cudaMemcpyHostToDevice, st)))
    return fail(e);
  if (nmodes > 0) {
    // slots 0..3 = mu^0..mu^6; the top-hat sum goes to slot 4 whatever l_max is
    k_sg_shells<<<(nmodes + 255) / 256, 256, 0, st>>>(d_modes, nmodes, d_acc, d_invw, n, nmain, wedge ? 1 : 0,
                                                      nbins, d_sacc);
    if ((e = cudaGetLastError())) return fail(e);
  }
  k_sg_finalize<<<1, 256, 0, st>>>(d_sacc, d_shell, d_sums, alpha_cfg, nbins, ell, wedge ? 1 : 0, d_out, d_wedges);
  if ((e = cudaGetLastError())) return fail(e);
  if ((e = cudaStreamSynchronize(st))) return fail(e);
  return YS_OK;
}

}  // namespace
}  // namespace ys

using namespace ys;

extern "C" ys_status ys_sum_gal(const ys_config* cfg, const ys_catalog* gal, const ys_catalog* ran, double* d_out,
                                double* d_wedges) {
  if (!cfg || !gal || !ran || !d_out) return YS_ERR_ARG;
  const ys_config& c = *cfg;
  if (c.n_mesh < 4 || c.n_mesh > 16384 || (c.n_mesh & 1)) return YS_ERR_ARG;
  if (!(c.box_len > 0) || !std::isfinite(c.box_len)) return YS_ERR_ARG;
  if (c.ell_max != 0 && c.ell_max != 2 && c.ell_max != 4 && c.ell_max != 6) return YS_ERR_ARG;
  if (c.n_bins <= 0 || c.n_bins > 4096 || !(c.dk > 0) || !(c.k_min >= 0)) return YS_ERR_ARG;
  for (const ys_catalog* k : {gal, ran})
    if (k->n < 0 || (k->n > 0 && (!k->x || !k->y || !k->z))) return YS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(c.stream);
  const ModeTable mt = build_modes(c);
  const int nmodes = (int)mt.modes.size();
  const bool wedge = d_wedges != nullptr;
  Scratch sc;
  SgMode* d_modes = nullptr;
  double *d_acc = nullptr, *d_sums = nullptr;
  SgPoint* d_pts = nullptr;
  const int64_t npts = gal->n + ran->n;
  cudaError_t e;
  if ((e = sc.get(d_modes, (size_t)nmodes)) || (e = sc.get(d_acc, (size_t)C_COUNT * 2 * std::max(1, nmodes))) ||
      (e = sc.get(d_sums, (size_t)SUM_COUNT)) || (e = sc.get(d_pts, (size_t)std::max<int64_t>(1, npts))))
    return fail(e);
  if (nmodes > 0 && (e = cudaMemcpyAsync(d_modes, mt.modes.data(), sizeof(SgMode) * nmodes, cudaMemcpyHostToDevice, st)))
    return fail(e);
  if ((e = cudaMemsetAsync(d_acc, 0, sizeof(double) * C_COUNT * 2 * std::max(1, nmodes), st)) ||
      (e = cudaMemsetAsync(d_sums, 0, sizeof(double) * SUM_COUNT, st)))
    return fail(e);
  const ys_catalog* cats[2] = {gal, ran};
  for (int k = 0; k < 2; ++k)
    if (cats[k]->n > 0) {
      const unsigned blocks = (unsigned)std::min<int64_t>(1024, (cats[k]->n + 255) / 256);
      k_sg_sums<<<blocks, 256, 0, st>>>(cats[k]->w, cats[k]->nbar, cats[k]->n, k, d_sums);
      if ((e = cudaGetLastError())) return fail(e);
    }
  int64_t off = 0;
  for (int k = 0; k < 2; ++k) {
    const ys_catalog& q = *cats[k];
    if (q.n > 0) {
      k_sg_points_cat<<<(unsigned)((q.n + 255) / 256), 256, 0, st>>>(
          q.x, q.y, q.z, q.w, q.n, k, d_sums, c.alpha, c.box_min[0], c.box_min[1], c.box_min[2], 1.0 / c.box_len,
          c.observer[0], c.observer[1], c.observer[2], d_pts + off);
      if ((e = cudaGetLastError())) return fail(e);
    }
    off += q.n;
  }
  if (nmodes > 0 && npts > 0 && (e = run_modes(c.ell_max, wedge, d_modes, nmodes, d_pts, nullptr, npts, d_acc, st)))
    return fail(e);
  return finish(mt, d_modes, d_acc, nullptr, c.n_mesh, d_sums, c.alpha, c.n_bins, c.ell_max, wedge, d_out, d_wedges,
                sc, st);
}

extern "C" ys_status ys_sum_grid(ys_plan* plan, double* d_out, double* d_wedges) {
  if (!plan || !d_out) return YS_ERR_ARG;
  Plan& p = plan->p;
  if (!p.assigned) return YS_ERR_STATE;
  const ys_config& c = p.cfg;
  cudaStream_t st = p.stream;
  const ModeTable mt = build_modes(c);
  const int nmodes = (int)mt.modes.size();
  const bool wedge = d_wedges != nullptr;
  const int64_t n3 = (int64_t)p.n * p.n * p.n;
  // the nodes go through in chunks of at most 2^26 (2 GB of points), each added into
  // the FP64 per-mode sums
  const int64_t chunk = std::min<int64_t>(n3, (int64_t)1 << 26);
  Scratch sc;
  SgMode* d_modes = nullptr;
  double* d_acc = nullptr;
  SgPoint* d_pts = nullptr;
  unsigned* d_count = nullptr;
  cudaError_t e;
  if ((e = sc.get(d_modes, (size_t)nmodes)) || (e = sc.get(d_acc, (size_t)C_COUNT * 2 * std::max(1, nmodes))) ||
      (e = sc.get(d_pts, (size_t)chunk)) || (e = sc.get(d_count, 1)))
    return fail(e);
  if (nmodes > 0 && (e = cudaMemcpyAsync(d_modes, mt.modes.data(), sizeof(SgMode) * nmodes, cudaMemcpyHostToDevice, st)))
    return fail(e);
  if ((e = cudaMemsetAsync(d_acc, 0, sizeof(double) * C_COUNT * 2 * std::max(1, nmodes), st))) return fail(e);
  // The interlaced pair is averaged: each mesh's nodes carry F / 2.
  const float scale = p.m == 2 ? 0.5f : 1.f;
  for (int j = 0; j < p.m; ++j)
    for (int64_t first = 0; first < n3 && nmodes > 0; first += chunk) {
      const int64_t cnt = std::min(chunk, n3 - first);
      if ((e = cudaMemsetAsync(d_count, 0, sizeof(unsigned), st))) return fail(e);
      k_sg_points_mesh<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(
          p.d_mesh + j * n3, p.n, j, first, cnt, c.box_min[0] - c.observer[0], c.box_min[1] - c.observer[1],
          c.box_min[2] - c.observer[2], p.H, scale, d_count, d_pts);
      if ((e = cudaGetLastError())) return fail(e);
      if ((e = run_modes(c.ell_max, wedge, d_modes, nmodes, d_pts, d_count, cnt, d_acc, st))) return fail(e);
    }
  return finish(mt, d_modes, d_acc, c.compensate ? p.d_invw : nullptr, p.n, p.d_sums, c.alpha, c.n_bins, c.ell_max,
                wedge, d_out, d_wedges, sc, st);
}
