// C ABI of the ystat library: plan creation (validation, FP64 host tables, device
// allocation), the assign / measure entry points, and the final Eqs. (6)-(8).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fft.cuh"
#include "ys_internal.h"

namespace ys {

template <int N> cudaError_t run_measure_n(Plan* const* lanes, int W, double* const* rows);
template <int N> int yz_grid_n(int ell, cudaError_t* err);
template <int N> size_t x_smem_n(int nbins, int nwb, int ell);

thread_local std::string g_last_cuda_error;
int yz_row_items(int n);

namespace {

ys_status cuda_fail(cudaError_t e) {
  g_last_cuda_error = cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? YS_ERR_OOM : YS_ERR_CUDA;
}

bool supported_n(int n) {
  static const int ok[] = {16, 32, 64, 96, 128, 192, 256, 384, 512, 768, 1024};
  for (int v : ok)
    if (v == n) return true;
  return false;
}

template <class T>
cudaError_t dalloc(Plan& p, T*& ptr, size_t count) {
  void* raw = nullptr;
  cudaError_t e = cudaMalloc(&raw, count * sizeof(T) + 16);
  if (e == cudaSuccess) {
    ptr = static_cast<T*>(raw);
    p.device_bytes += count * sizeof(T) + 16;
  }
  return e;
}

template <class T>
void dfree(T*& ptr) {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
}

void free_all(Plan& p) {
  dfree(p.d_tw); dfree(p.d_nodes); dfree(p.d_rel); dfree(p.d_invw); dfree(p.d_phase);
  dfree(p.d_col_off); dfree(p.d_pencil); dfree(p.d_lut); dfree(p.d_shell);
  dfree(p.d_mesh); dfree(p.d_z); dfree(p.d_sync); dfree(p.d_g); dfree(p.d_acc); dfree(p.d_sums); dfree(p.d_result);
  dfree(p.d_tile_count); dfree(p.d_tile_off); dfree(p.d_tile_cur); dfree(p.d_rec);
  dfree(p.d_stage);
  dfree(p.d_rmesh); dfree(p.d_rsums);
  p.device_bytes = 0;
}

// Result row: [k_mean | n_modes | p0 | p2 | p4 | alpha, I, S/I, n_out, timeout] and, for
// l_max = 6, p6 after the five scalars (so rows of l_max <= 4 plans keep their layout).
// One CTA per lane (plans of one configuration measured together); lane l's shell
// sums, catalogue sums and flag are its own, the shell table is the configuration's.
struct FinMulti {
  const double* acc[YZ_MAX_LANES];
  const double* sums[YZ_MAX_LANES];
  const int* flags[YZ_MAX_LANES];
  double* res[YZ_MAX_LANES];
};

__global__ void k_finalize(const __grid_constant__ FinMulti fm, const double* __restrict__ shell, double alpha_cfg,
                           int nbins, int ell) {
  const double* __restrict__ acc = fm.acc[blockIdx.x];
  const double* __restrict__ sums = fm.sums[blockIdx.x];
  const int* __restrict__ flags = fm.flags[blockIdx.x];
  double* __restrict__ res = fm.res[blockIdx.x];
  const double alpha = alpha_cfg >= 0.0 ? alpha_cfg : sums[SUM_WG] / sums[SUM_WR];
  const double I = alpha * sums[SUM_WR2N];
  const double S = sums[SUM_WG2] + alpha * alpha * sums[SUM_WR2];
  const double nan = __longlong_as_double(0x7ff8000000000000ULL);
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    const double nm = shell[b];
    double km = nan, p0 = nan, p2 = nan, p4 = nan, p6 = nan;
    if (nm > 0.0) {
      km = shell[nbins + b] / nm;
      const double m0 = acc[b] / nm, m2 = acc[nbins + b] / nm, m4 = acc[2 * nbins + b] / nm;
      // Eqs. (6)-(8), shot noise subtracted from the monopole only (Eq. 3).
      p0 = (m0 - S) / I;
      if (ell >= 2) p2 = 2.5 / I * (3.0 * m2 - m0);
      if (ell >= 4) p4 = 1.125 / I * (35.0 * m4 - 30.0 * m2 + 3.0 * m0);
      // l = 6, the same step one order up: 13/I <Re A_0 L_6^*>, L_6(mu) =
      // (231 mu^6 - 315 mu^4 + 105 mu^2 - 5) / 16 written with the mu-power sums.
      if (ell >= 6) p6 = 0.8125 / I * (231.0 * acc[3 * nbins + b] / nm - 315.0 * m4 + 105.0 * m2 - 5.0 * m0);
    }
    res[b] = km;
    res[nbins + b] = nm;
    res[2 * nbins + b] = p0;
    res[3 * nbins + b] = p2;
    res[4 * nbins + b] = p4;
    if (ell >= 6) res[5 * nbins + 5 + b] = p6;
  }
  if (threadIdx.x == 0) {
    res[5 * nbins + 0] = alpha;
    res[5 * nbins + 1] = I;
    res[5 * nbins + 2] = S / I;
    res[5 * nbins + 3] = sums[SUM_BAD];
    res[5 * nbins + 4] = (double)flags[0];
  }
}

size_t x_smem_for(int n, int nbins, int nwb, int ell) {
  switch (n) {
    case 16: return x_smem_n<16>(nbins, nwb, ell);
    case 32: return x_smem_n<32>(nbins, nwb, ell);
    case 64: return x_smem_n<64>(nbins, nwb, ell);
    case 96: return x_smem_n<96>(nbins, nwb, ell);
    case 128: return x_smem_n<128>(nbins, nwb, ell);
    case 192: return x_smem_n<192>(nbins, nwb, ell);
    case 256: return x_smem_n<256>(nbins, nwb, ell);
    case 384: return x_smem_n<384>(nbins, nwb, ell);
    case 512: return x_smem_n<512>(nbins, nwb, ell);
    case 768: return x_smem_n<768>(nbins, nwb, ell);
    default: return x_smem_n<1024>(nbins, nwb, ell);
  }
}

// 2D tensor map over the grouped transforms d_g: rows = (mesh, group, x), columns =
// 2 np_pad floats (np_pad float2 pencils); box = (2 P floats, x_box_rows(N) rows, a
// divisor of N of at most 256).
ys_status make_gmap(Plan& p) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || !fn || q != cudaDriverEntryPointSuccess) {
    g_last_cuda_error = "cuTensorMapEncodeTiled not available";
    return YS_ERR_CUDA;
  }
  auto encode = reinterpret_cast<CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                              CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                              CUtensorMapFloatOOBfill)>(fn);
  const int P = p.x_pencils;
  const cuuint64_t dims[2] = {(cuuint64_t)2 * p.np_pad, (cuuint64_t)p.m * p.ng * p.n};
  const cuuint64_t strides[1] = {(cuuint64_t)2 * p.np_pad * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * P), (cuuint32_t)x_box_rows(p.n)};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(&p.gmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, p.d_g, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    g_last_cuda_error = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return YS_ERR_CUDA;
  }
  return YS_OK;
}

}  // namespace

ys_status set_x_pencils(Plan& p, int pencils) {
  if (pencils != k3_pencils(p.n) && pencils != k3_pencils_alt(p.n)) return YS_ERR_ARG;
  if (pencils == p.x_pencils) return YS_OK;
  const int old = p.x_pencils;
  p.x_pencils = pencils;
  if (p.np > 0) {
    ys_status st = make_gmap(p);
    if (st != YS_OK) {
      p.x_pencils = old;
      make_gmap(p);
      return st;
    }
  }
  if (p.measure_exec) {
    cudaGraphExecDestroy(p.measure_exec);
    p.measure_exec = nullptr;
  }
  return YS_OK;
}

namespace {

// FP64 host tables (shells, pencils, windows, phases, twiddles, node positions).
ys_status build_tables(Plan& p) {
  const ys_config& c = p.cfg;
  const int n = p.n;
  const double L = c.box_len;
  p.H = L / n;
  p.kf = 2.0 * M_PI / L;
  const double knyq = p.kf * n / 2.0;
  // shell index per integer |m|^2 (only |m|^2 < (n/2)^2 can satisfy |k| < k_Nyquist)
  const int n2max = (n / 2) * (n / 2);
  std::vector<short> lut(n2max, -1);
  int n2_hi = 0;
  for (int n2 = 1; n2 < n2max; ++n2) {
    const double kmag = p.kf * std::sqrt((double)n2);
    if (!(kmag < knyq)) continue;
    const double b = std::floor((kmag - c.k_min) / c.dk);
    if (b >= 0 && b < c.n_bins) {
      lut[n2] = (short)b;
      n2_hi = n2 + 1;
    }
  }
  p.n2_hi = n2_hi;
  // pencils (k_y, k_z), k_z >= 0, k_y^2 + k_z^2 < n2_hi; column k_z holds |k_y| <= kymax
  std::vector<int> col_off;
  std::vector<short2> pen;
  int nzc = 0;
  while (n2_hi > 0 && nzc * nzc < n2_hi) ++nzc;
  col_off.push_back(0);
  for (int kz = 0; kz < nzc; ++kz) {
    int kymax = 0;
    while ((kymax + 1) * (kymax + 1) + kz * kz < n2_hi) ++kymax;
    for (int ky = -kymax; ky <= kymax; ++ky) pen.push_back(make_short2((short)ky, (short)kz));
    col_off.push_back((int)pen.size());
  }
  p.nzc = nzc;
  p.np = (int)pen.size();
  // pad to whole x-stage pencil blocks of either size with pencils that match no
  // shell (k_z = -1)
  const int xp = std::max(k3_pencils(n), k3_pencils_alt(n));
  p.x_pencils = k3_pencils(n);
  p.np_pad = std::max(xp, (p.np + xp - 1) / xp * xp);
  while ((int)pen.size() < p.np_pad) pen.push_back(make_short2(0, -1));
  // mode count and sum |k| per shell (half grid, weight 2 for 0 < k_z < n/2)
  std::vector<double> shell(2 * c.n_bins, 0.0);
  for (int kz = 0; kz < nzc; ++kz) {
    const int kymax = (col_off[kz + 1] - col_off[kz] - 1) / 2;
    const double w = kz == 0 ? 1.0 : 2.0;
    for (int ky = -kymax; ky <= kymax; ++ky)
      for (int mx = -n / 2 + 1; mx < n / 2; ++mx) {
        const int n2 = mx * mx + ky * ky + kz * kz;
        if (n2 >= n2_hi || n2 <= 0) continue;
        const int b = lut[n2];
        if (b < 0) continue;
        shell[b] += w;
        shell[c.n_bins + b] += w * p.kf * std::sqrt((double)n2);
      }
  }
  // per-axis window compensation and interlacing phase by FFT index
  const int pw = c.assign;  // NGP 1, CIC 2, TSC 3
  std::vector<float> invw(n);
  std::vector<float2> phase(n), tw(n);
  for (int i = 0; i < n; ++i) {
    const int m = i <= n / 2 ? i : i - n;
    const double x = M_PI * m / n;
    double W = 1.0;
    if (m != 0) W = std::pow(std::sin(x) / x, pw);
    invw[i] = c.compensate ? (float)(1.0 / W) : 1.0f;
    phase[i] = make_float2((float)std::cos(x), (float)-std::sin(x));
  }
  // stage-major twiddles (fft_tw_offset): exp(-2 pi i r k / (N_s R_s)) per stage
  for (int st = 1; st < fft_nstages(n); ++st) {
    const int ns = fft_ns_before(n, st), rad = fft_radix(n, st), off = fft_tw_offset(n, st);
    for (int k = 0; k < ns; ++k)
      for (int r = 1; r < rad; ++r) {
        const double t = -2.0 * M_PI * r * k / ((double)ns * rad);
        tw[off + k * (rad - 1) + r - 1] = make_float2((float)std::cos(t), (float)std::sin(t));
      }
  }
  // node positions (hi, lo) for i in [-1, n + 1], and node - observer per mesh
  std::vector<float2> nodes(3 * (n + 3));
  for (int a = 0; a < 3; ++a)
    for (int i = -1; i <= n + 1; ++i) {
      const double v = c.box_min[a] + i * p.H;
      const float hi = (float)v;
      nodes[a * (n + 3) + i + 1] = make_float2(hi, (float)(v - (double)hi));
    }
  std::vector<float> rel((size_t)p.m * 3 * n);
  for (int j = 0; j < p.m; ++j)
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < n; ++i) {
        const double s = j == 1 ? 0.5 : 0.0;
        rel[((size_t)j * 3 + a) * n + i] = (float)(c.box_min[a] + (i + s) * p.H - c.observer[a]);
      }
  cudaError_t e;
#define YS_UP(dst, vec)                                                                                 \
  do {                                                                                                  \
    if ((e = dalloc(p, dst, std::max<size_t>(1, vec.size())))) return cuda_fail(e);                     \
    if (!vec.empty() &&                                                                                 \
        (e = cudaMemcpy(dst, vec.data(), vec.size() * sizeof(vec[0]), cudaMemcpyHostToDevice)))         \
      return cuda_fail(e);                                                                              \
  } while (0)
  YS_UP(p.d_lut, lut);
  YS_UP(p.d_col_off, col_off);
  YS_UP(p.d_pencil, pen);
  YS_UP(p.d_shell, shell);
  YS_UP(p.d_invw, invw);
  YS_UP(p.d_phase, phase);
  YS_UP(p.d_tw, tw);
  YS_UP(p.d_nodes, nodes);
  YS_UP(p.d_rel, rel);
#undef YS_UP
  return YS_OK;
}

bool catalog_ok(const ys_catalog* k) {
  if (!k || k->n < 0) return false;
  if (k->n > 0 && (!k->x || !k->y || !k->z)) return false;
  return true;
}

}  // namespace

ys_status ensure_particles(Plan& p, int64_t total) {
  if (total <= p.part_cap) return YS_OK;
  cudaError_t e;
  if (p.d_rec) {
    if ((e = cudaStreamSynchronize(p.stream))) return cuda_fail(e);
    p.device_bytes -= (size_t)p.rec_cap * sizeof(float4) + 16;
    dfree(p.d_rec);
  }
  // records per particle: up to 2 tiles per axis that has more than one tile, for
  // any scatter-tile shape the tuner may switch to
  int factor = 1;
  for (const auto& t : kTileCandidates) {
    int f = 1;
    for (int a = 0; a < 3; ++a) f *= std::min(t[a], p.n) < p.n ? 2 : 1;
    factor = std::max(factor, f);
  }
  p.part_cap = total;
  p.rec_cap = total * factor;
  if ((e = dalloc(p, p.d_rec, (size_t)p.rec_cap))) return cuda_fail(e);
  return YS_OK;
}

void set_tiles(Plan& p, int tx, int ty, int tz) {
  const int t[3] = {tx, ty, tz};
  p.ntiles = 1;
  for (int a = 0; a < 3; ++a) {
    p.geom.tdim[a] = std::min(t[a], p.n);
    p.geom.tiles[a] = p.n / p.geom.tdim[a];
    p.ntiles *= p.geom.tiles[a];
  }
}

// Lead D of the y,z ring: the column items of plane p are claimed D planes after its
// row items, and must not be claimed before those finish (a claimed item that waits
// idles its CTA).  Between the two claims the grid works through about
// D * W_plane - (grid - NZ) * w_row of other items, with W_plane = NZ w_row + NY w_col
// the work of one plane's items in FFT-line units (a row item: R rows x field pairs,
// plus field construction; a column item: its basis fields plus the fold).
int ring_lead_for(const Plan& p, int grid, int pct) {
  const int nz = yz_row_items(p.n), ny = std::max(1, p.nzc);
  const double rows = (double)p.n / nz;
  const double w_row = rows * ((p.nb + 1) / 2) * 1.3, w_col = p.nb * 1.2;
  const double plane = nz * w_row + ny * w_col;
  const double base = std::ceil(std::max(0, grid - nz) * w_row / plane) + 1.0;
  return std::max(2, (int)std::ceil(base * pct / 100.0));
}

void set_yz_grid(Plan& p, int grid, int lead_pct) {
  p.yz_grid = std::max(1, std::min(grid, p.yz_grid_max));
  if (lead_pct > 0) p.ring_lead_pct = lead_pct;
  const int slots_max = p.ring_slots_cap > 0 ? p.ring_slots_cap : p.m * p.n;
  p.ring_lead = std::min(ring_lead_for(p, p.yz_grid, p.ring_lead_pct), std::max(1, slots_max - 2));
  p.ring_slots = std::min(p.m * p.n, p.ring_lead + 2);
}

LaunchScope::LaunchScope(Plan& plan, int c) : p(plan), cls(c) {
  if (p.capturing) {
    ++p.measure_launches[c];
    return;
  }
  ++p.launches[c];
  if (p.profiling) {
    for (cudaEvent_t* ev : {&a, &b}) {
      if (!p.event_pool.empty()) {
        *ev = p.event_pool.back();
        p.event_pool.pop_back();
      } else if (cudaEventCreate(ev) != cudaSuccess) {
        *ev = nullptr;
      }
    }
    if (a && b) cudaEventRecord(a, p.stream);
  }
}

LaunchScope::~LaunchScope() {
  if (a && b) {
    cudaEventRecord(b, p.stream);
    p.pending.push_back({a, b, cls});
  }
}

cudaError_t launch_finalize(Plan* const* lanes, int W, double* const* rows) {
  Plan& p = *lanes[0];
  FinMulti fm{};
  for (int l = 0; l < W; ++l) {
    Plan& q = *lanes[l];
    fm.acc[l] = q.d_acc;
    fm.sums[l] = q.d_sums;
    fm.flags[l] = q.d_sync + 2 * q.m * q.n + 1;
    fm.res[l] = rows[l];
  }
  LaunchScope ls(p, 7);
  k_finalize<<<W, 256, 0, p.stream>>>(fm, p.d_shell, p.cfg.alpha, p.cfg.n_bins, p.ell);
  return cudaGetLastError();
}

// Row items per plane of the y,z kernel (N / rows per item; mirrors YZ<N, ELL>::R).
int yz_row_items(int n) {
  const int E = (n & (n - 1)) == 0 ? 8 : 12;  // fft_elems
  const int lpp = 256 / (n / E);
  const int base = n >= 512 ? 8 : 16;
  const int r = lpp > base ? std::min(lpp, n) : base;
  return n / r;
}

int yz_grid_for(Plan& p, cudaError_t* err) {
  switch (p.n) {
    case 16: return yz_grid_n<16>(p.ell, err);
    case 32: return yz_grid_n<32>(p.ell, err);
    case 64: return yz_grid_n<64>(p.ell, err);
    case 96: return yz_grid_n<96>(p.ell, err);
    case 128: return yz_grid_n<128>(p.ell, err);
    case 192: return yz_grid_n<192>(p.ell, err);
    case 256: return yz_grid_n<256>(p.ell, err);
    case 384: return yz_grid_n<384>(p.ell, err);
    case 512: return yz_grid_n<512>(p.ell, err);
    case 768: return yz_grid_n<768>(p.ell, err);
    case 1024: return yz_grid_n<1024>(p.ell, err);
    default: *err = cudaErrorInvalidValue; return 0;
  }
}

cudaError_t launch_measure_lanes(Plan* const* lanes, int W, double* const* rows) {
  if (W < 1 || W > YZ_MAX_LANES) return cudaErrorInvalidValue;
  switch (lanes[0]->n) {
    case 16: return run_measure_n<16>(lanes, W, rows);
    case 32: return run_measure_n<32>(lanes, W, rows);
    case 64: return run_measure_n<64>(lanes, W, rows);
    case 96: return run_measure_n<96>(lanes, W, rows);
    case 128: return run_measure_n<128>(lanes, W, rows);
    case 192: return run_measure_n<192>(lanes, W, rows);
    case 256: return run_measure_n<256>(lanes, W, rows);
    case 384: return run_measure_n<384>(lanes, W, rows);
    case 512: return run_measure_n<512>(lanes, W, rows);
    case 768: return run_measure_n<768>(lanes, W, rows);
    case 1024: return run_measure_n<1024>(lanes, W, rows);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_measure(Plan& p) {
  Plan* lane = &p;
  double* row = p.d_result;
  return launch_measure_lanes(&lane, 1, &row);
}

}  // namespace ys

using ys::Plan;

extern "C" {

const char* ys_status_string(ys_status s) {
  switch (s) {
    case YS_OK: return "ok";
    case YS_ERR_ARG: return "invalid argument";
    case YS_ERR_OOM: return "device allocation failed";
    case YS_ERR_CUDA: return "CUDA error";
    case YS_ERR_TIMEOUT: return "device wait timed out";
    case YS_ERR_UNSUPPORTED: return "unsupported configuration";
    case YS_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char* ys_last_cuda_error(void) { return ys::g_last_cuda_error.c_str(); }

ys_status ys_plan_create(const ys_config* cfg, ys_plan** out) {
  if (!cfg || !out) return YS_ERR_ARG;
  *out = nullptr;
  const ys_config& c = *cfg;
  if (!ys::supported_n(c.n_mesh)) return YS_ERR_UNSUPPORTED;
  if (c.ell_max == 6 && c.n_mesh > 512) {  // the column item's 29 lines exceed shared memory
    ys::g_last_cuda_error = "l_max = 6 is supported up to 512^3";
    return YS_ERR_UNSUPPORTED;
  }
  if (!(c.box_len > 0) || !std::isfinite(c.box_len)) return YS_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(c.box_min[a]) || !std::isfinite(c.observer[a])) return YS_ERR_ARG;
  if (c.assign < YS_NGP || c.assign > YS_TSC) return YS_ERR_ARG;
  if (c.interlace != 0 && c.interlace != 1) return YS_ERR_ARG;
  if (c.compensate != 0 && c.compensate != 1) return YS_ERR_ARG;
  if (c.ell_max != 0 && c.ell_max != 2 && c.ell_max != 4 && c.ell_max != 6) return YS_ERR_ARG;
  if (c.n_bins <= 0 || c.n_bins > 4096 || !(c.dk > 0) || !(c.k_min >= 0)) return YS_ERR_ARG;
  if (c.max_particles < 0) return YS_ERR_ARG;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    ys::g_last_cuda_error = e != cudaSuccess ? cudaGetErrorString(e) : "no CUDA device";
    return YS_ERR_CUDA;
  }
  {  // the x stage keeps every shell's sums in shared memory
    int dev = 0, smem_max = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) {
      ys::g_last_cuda_error = cudaGetErrorString(e);
      return YS_ERR_CUDA;
    }
    if (ys::x_smem_for(c.n_mesh, c.n_bins, 1, c.ell_max) > (size_t)smem_max) {
      ys::g_last_cuda_error = std::to_string(c.n_bins) + " shells do not fit the shared memory of the " +
                              std::to_string(c.n_mesh) + "^3 x stage";
      return YS_ERR_UNSUPPORTED;
    }
  }
  ys_plan* h = new (std::nothrow) ys_plan;
  if (!h) return YS_ERR_OOM;
  Plan& p = h->p;
  p.cfg = c;
  p.stream = static_cast<cudaStream_t>(c.stream);
  p.n = c.n_mesh;
  p.m = c.interlace ? 2 : 1;
  p.ell = c.ell_max;
  p.kind = c.assign;
  p.nb = p.ell == 0 ? 1 : (p.ell == 2 ? 7 : (p.ell == 4 ? 16 : 29));
  p.ng = p.ell == 0 ? 1 : (p.ell == 2 ? 4 : (p.ell == 4 ? 9 : 16));
  p.row_len = ys::result_row_len(c.n_bins, p.ell);
  const int n = p.n;
  ys::Geom& g = p.geom;
  g.n = n;
  g.inv_h = (float)(n / c.box_len);
  for (int a = 0; a < 3; ++a) g.bmin[a] = (float)c.box_min[a];
  // tile counters sized for every scatter-tile candidate the tuner may pick
  p.ntiles_max = 0;
  for (const auto& t : ys::kTileCandidates) {
    ys::set_tiles(p, t[0], t[1], t[2]);
    p.ntiles_max = std::max(p.ntiles_max, p.ntiles);
  }
  ys::set_tiles(p, ys::TILE_X, ys::TILE_Y, ys::TILE_Z);
  // a mesh set of at most 64 MB (half of L2) can stay in L2 during the direct assignment
  p.direct_ok = (size_t)p.m * n * n * n * sizeof(float) <= (64u << 20);
  ys_status st = ys::build_tables(p);
  if (st != YS_OK) {
    ys::free_all(p);
    delete h;
    return st;
  }
  const size_t n3 = (size_t)n * n * n;
  // y,z-stage ring: the column items of a plane trail its row items by D planes, and a
  // slot is rewritten S = D + 2 planes later; D covers one grid's worth of items.
  p.yz_grid_max = ys::yz_grid_for(p, &e);
  if (e) {
    st = ys::cuda_fail(e);
    ys::free_all(p);
    delete h;
    return st;
  }
  // ring sized for the largest grid and lead the tuner may pick
  ys::set_yz_grid(p, p.yz_grid_max, ys::kRingLeadPctMax);
  p.ring_slots_cap = p.ring_slots;
  ys::set_yz_grid(p, p.yz_grid_max, 100);
  const size_t slot = (size_t)2 * ((p.nb + 1) / 2) * std::max(1, p.nzc) * n;  // field pairs interleaved
  if ((e = ys::dalloc(p, p.d_mesh, p.m * n3)) || (e = ys::dalloc(p, p.d_z, slot * p.ring_slots_cap)) ||
      (e = ys::dalloc(p, p.d_sync, (size_t)2 * p.m * n + 2)) ||
      (e = ys::dalloc(p, p.d_g, (size_t)p.m * p.ng * n * std::max(1, p.np_pad))) ||
      (e = ys::dalloc(p, p.d_acc, (size_t)4 * c.n_bins)) || (e = ys::dalloc(p, p.d_sums, (size_t)ys::SUM_COUNT)) ||
      (e = ys::dalloc(p, p.d_result, (size_t)p.row_len)) ||
      (e = ys::dalloc(p, p.d_tile_count, (size_t)p.ntiles_max)) ||
      (e = ys::dalloc(p, p.d_tile_off, (size_t)p.ntiles_max + 1)) ||
      (e = ys::dalloc(p, p.d_tile_cur, (size_t)p.ntiles_max))) {
    st = ys::cuda_fail(e);
    ys::free_all(p);
    delete h;
    return st;
  }
  if (p.np > 0 && (st = ys::make_gmap(p)) != YS_OK) {
    ys::free_all(p);
    delete h;
    return st;
  }
  if (c.max_particles > 0 && (st = ys::ensure_particles(p, c.max_particles)) != YS_OK) {
    ys::free_all(p);
    delete h;
    return st;
  }
  p.h_result.assign((size_t)p.row_len, 0.0);
  if (cudaStreamCreateWithFlags(&p.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    p.cap_stream = nullptr;
  }
  *out = h;
  return YS_OK;
}

size_t ys_plan_device_bytes(const ys_plan* plan) { return plan ? plan->p.device_bytes : 0; }

ys_status ys_assign(ys_plan* plan, const ys_catalog* gal, const ys_catalog* ran) {
  if (!plan || !ys::catalog_ok(gal) || !ys::catalog_ok(ran)) return YS_ERR_ARG;
  Plan& p = plan->p;
  ys_status st = ys::ensure_particles(p, gal->n + ran->n);
  if (st != YS_OK) return st;
  cudaError_t e = ys::launch_assign(p, *gal, *ran);
  if (e) return ys::cuda_fail(e);
  p.assigned = true;
  return YS_OK;
}

ys_status ys_randoms_cache(ys_plan* plan, const ys_catalog* ran) {
  if (!plan || !ys::catalog_ok(ran)) return YS_ERR_ARG;
  Plan& p = plan->p;
  ys_status st = ys::ensure_particles(p, ran->n);
  if (st != YS_OK) return st;
  cudaError_t e;
  const size_t n3 = (size_t)p.n * p.n * p.n;
  if (!p.d_rmesh && ((e = ys::dalloc(p, p.d_rmesh, p.m * n3)) || (e = ys::dalloc(p, p.d_rsums, 3))))
    return ys::cuda_fail(e);
  // The randoms go through the assignment as a catalogue of weight +w, into the kept
  // mesh instead of the plan's; their FP64 sums are taken separately.
  const ys_catalog none{nullptr, nullptr, nullptr, nullptr, nullptr, 0};
  float* mesh = p.d_mesh;
  p.d_mesh = p.d_rmesh;
  e = ys::launch_assign(p, *ran, none);
  p.d_mesh = mesh;
  if (!e) e = ys::launch_random_sums(p, *ran, p.d_rsums);
  if (e) return ys::cuda_fail(e);
  p.randoms_cached = true;
  p.assigned = false;  // the plan's catalogue sums were used as scratch
  return YS_OK;
}

ys_status ys_assign_cached(ys_plan* plan, const ys_catalog* gal) {
  if (!plan || !ys::catalog_ok(gal)) return YS_ERR_ARG;
  Plan& p = plan->p;
  if (!p.randoms_cached) return YS_ERR_STATE;
  ys_status st = ys::ensure_particles(p, gal->n);
  if (st != YS_OK) return st;
  const ys_catalog none{nullptr, nullptr, nullptr, nullptr, nullptr, 0};
  cudaError_t e = ys::launch_assign(p, *gal, none, p.d_rmesh, p.d_rsums);
  if (e) return ys::cuda_fail(e);
  p.assigned = true;
  return YS_OK;
}

ys_status ys_assign_noalloc(ys_plan* plan, const ys_catalog* gal, const ys_catalog* ran) {
  if (!plan || !ys::catalog_ok(gal) || !ys::catalog_ok(ran)) return YS_ERR_ARG;
  std::string why;
  const ys_status st = ys::assign_noalloc(plan->p, *gal, *ran, why);
  if (st != YS_OK) ys::g_last_cuda_error = why;
  return st;
}

ys_status ys_measure_multipoles_async(ys_plan* plan, double* d_out) {
  if (!plan) return YS_ERR_ARG;
  Plan& p = plan->p;
  if (!p.assigned) return YS_ERR_STATE;
  cudaError_t e = cudaSuccess;
  if (!p.profiling && p.cap_stream && !p.measure_exec) {
    // Capture the measurement sequence once; every later call replays it.
    cudaStream_t user = p.stream;
    p.stream = p.cap_stream;
    p.capturing = true;
    for (int c = 0; c < YS_NUM_KERNEL_CLASSES; ++c) p.measure_launches[c] = 0;
    e = cudaStreamBeginCapture(p.cap_stream, cudaStreamCaptureModeThreadLocal);
    cudaError_t e2 = cudaSuccess;
    if (!e) {
      e2 = ys::launch_measure(p);
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(p.cap_stream, &graph);
      if (!e && !e2) e = cudaGraphInstantiate(&p.measure_exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
    }
    p.capturing = false;
    p.stream = user;
    if (e || e2 || !p.measure_exec) {  // no graph: launch directly from now on
      cudaGetLastError();
      if (p.measure_exec) cudaGraphExecDestroy(p.measure_exec);
      p.measure_exec = nullptr;
      cudaStreamDestroy(p.cap_stream);
      p.cap_stream = nullptr;
    }
    e = cudaSuccess;
  }
  if (!p.profiling && p.measure_exec) {
    e = cudaGraphLaunch(p.measure_exec, p.stream);
    if (e) return ys::cuda_fail(e);
    for (int c = 0; c < YS_NUM_KERNEL_CLASSES; ++c) p.launches[c] += p.measure_launches[c];
  } else {
    e = ys::launch_measure(p);
    if (e) return ys::cuda_fail(e);
  }
  if (d_out) {
    e = cudaMemcpyAsync(d_out, p.d_result, sizeof(double) * p.row_len, cudaMemcpyDeviceToDevice, p.stream);
    if (e) return ys::cuda_fail(e);
  }
  return YS_OK;
}

ys_status ys_measure_multipoles(ys_plan* plan, ys_result* out) {
  if (!plan || !out) return YS_ERR_ARG;
  Plan& p = plan->p;
  ys_status st = ys_measure_multipoles_async(plan, nullptr);
  if (st != YS_OK) return st;
  const int nb = p.cfg.n_bins;
  cudaError_t e = cudaMemcpyAsync(p.h_result.data(), p.d_result, sizeof(double) * p.row_len,
                                  cudaMemcpyDeviceToHost, p.stream);
  if (e) return ys::cuda_fail(e);
  if ((e = cudaStreamSynchronize(p.stream))) return ys::cuda_fail(e);
  const double* r = p.h_result.data();
  double* dst[5] = {out->k_mean, out->n_modes, out->p0, out->p2, out->p4};
  for (int q = 0; q < 5; ++q)
    if (dst[q]) std::memcpy(dst[q], r + (size_t)q * nb, sizeof(double) * nb);
  if (out->p6) {
    if (p.ell >= 6) std::memcpy(out->p6, r + (size_t)5 * nb + 5, sizeof(double) * nb);
    else for (int b = 0; b < nb; ++b) out->p6[b] = std::nan("");
  }
  out->alpha = r[5 * nb + 0];
  out->norm_I = r[5 * nb + 1];
  out->shot_noise = r[5 * nb + 2];
  if (r[5 * nb + 4] != 0) return YS_ERR_TIMEOUT;
  return r[5 * nb + 3] > 0 ? YS_ERR_ARG : YS_OK;
}

ys_status ys_estimate_host(ys_plan* plan, const ys_catalog* gal, const ys_catalog* ran, ys_result* out) {
  if (!plan || !ys::catalog_ok(gal) || !ys::catalog_ok(ran) || !out) return YS_ERR_ARG;
  Plan& p = plan->p;
  const int64_t need = 5 * (gal->n + ran->n);
  cudaError_t e;
  if (need > p.stage_cap) {
    if (p.d_stage) {
      if ((e = cudaStreamSynchronize(p.stream))) return ys::cuda_fail(e);
      p.device_bytes -= (size_t)p.stage_cap * sizeof(float) + 16;
      ys::dfree(p.d_stage);
    }
    if ((e = ys::dalloc(p, p.d_stage, (size_t)need))) return ys::cuda_fail(e);
    p.stage_cap = need;
  }
  // The copies are spread over the plan's stream and up to kCopyStreams more, so that
  // several copy engines run at once; the plan's stream waits for all of them.
  int nstreams = 1;
  if (!p.copy_event[0]) {
    bool ok = cudaEventCreateWithFlags(&p.copy_event[0], cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < Plan::kCopyStreams; ++k)
      ok = cudaStreamCreateWithFlags(&p.copy_stream[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&p.copy_event[k + 1], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) cudaGetLastError();
  }
  while (nstreams <= Plan::kCopyStreams && p.copy_stream[nstreams - 1] && p.copy_event[nstreams]) ++nstreams;
  if (!p.copy_event[0]) nstreams = 1;
  cudaStream_t streams[Plan::kCopyStreams + 1] = {p.stream};
  for (int k = 1; k < nstreams; ++k) streams[k] = p.copy_stream[k - 1];
  if (nstreams > 1) {
    if ((e = cudaEventRecord(p.copy_event[0], p.stream))) return ys::cuda_fail(e);
    for (int k = 1; k < nstreams; ++k)
      if ((e = cudaStreamWaitEvent(streams[k], p.copy_event[0], 0))) return ys::cuda_fail(e);
  }
  int next = 0;
  ys_catalog dev[2];
  const ys_catalog* src[2] = {gal, ran};
  float* cursor = p.d_stage;
  for (int c = 0; c < 2; ++c) {
    const ys_catalog& s = *src[c];
    ys_catalog& d = dev[c];
    d.n = s.n;
    const float* in[5] = {s.x, s.y, s.z, s.w, s.nbar};
    const float** outp[5] = {&d.x, &d.y, &d.z, &d.w, &d.nbar};
    for (int q = 0; q < 5; ++q) {
      // n-bar enters only through the randoms (I = alpha sum_r w^2 n-bar)
      if (!in[q] || s.n == 0 || (q == 4 && c == 0)) {
        *outp[q] = (q < 3) ? cursor : nullptr;
        continue;
      }
      if ((e = cudaMemcpyAsync(cursor, in[q], sizeof(float) * s.n, cudaMemcpyHostToDevice,
                               streams[next++ % nstreams])))
        return ys::cuda_fail(e);
      *outp[q] = cursor;
      cursor += s.n;
    }
  }
  for (int k = 1; k < nstreams; ++k) {
    if ((e = cudaEventRecord(p.copy_event[k], streams[k]))) return ys::cuda_fail(e);
    if ((e = cudaStreamWaitEvent(p.stream, p.copy_event[k], 0))) return ys::cuda_fail(e);
  }
  ys_status st = ys_assign(plan, &dev[0], &dev[1]);
  if (st != YS_OK) return st;
  return ys_measure_multipoles(plan, out);
}

ys_status ys_plan_destroy(ys_plan* plan) {
  if (!plan) return YS_OK;
  Plan& p = plan->p;
  if (p.stream) cudaStreamSynchronize(p.stream);
  else cudaDeviceSynchronize();
  if (p.measure_exec) cudaGraphExecDestroy(p.measure_exec);
  if (p.cap_stream) cudaStreamDestroy(p.cap_stream);
  for (cudaStream_t s : p.copy_stream)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t ev : p.copy_event)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : p.pending) {
    cudaEventDestroy(ev.a);
    cudaEventDestroy(ev.b);
  }
  for (cudaEvent_t ev : p.event_pool) cudaEventDestroy(ev);
  ys::free_all(p);
  delete plan;
  return YS_OK;
}

ys_status ys_plan_set_fault_injection(ys_plan* plan, int64_t wait_limit_ns, int32_t skip_plane) {
  if (!plan) return YS_ERR_ARG;
  Plan& p = plan->p;
  if (skip_plane < -1 || skip_plane >= p.m * p.n) return YS_ERR_ARG;
  const long long limit = wait_limit_ns > 0 ? (long long)wait_limit_ns : 1000000000LL;
  if (limit > 10000000000LL) return YS_ERR_ARG;
  if (p.stream) cudaStreamSynchronize(p.stream);
  p.yz_wait_ns = limit;
  p.fault_skip_plane = skip_plane;
  // the captured measurement graph holds the old kernel parameters: capture again
  if (p.measure_exec) {
    cudaGraphExecDestroy(p.measure_exec);
    p.measure_exec = nullptr;
  }
  return YS_OK;
}

ys_status ys_plan_set_direct_assign(ys_plan* plan, int enable) {
  if (!plan) return YS_ERR_ARG;
  Plan& p = plan->p;
  if (enable && !p.direct_ok) return YS_ERR_UNSUPPORTED;
  p.direct_assign = enable != 0;
  return YS_OK;
}

ys_status ys_plan_copy_mesh(ys_plan* plan, float* dst, int64_t count) {
  if (!plan || !dst) return YS_ERR_ARG;
  Plan& p = plan->p;
  const int64_t total = (int64_t)p.m * p.n * p.n * p.n;
  if (count < total) return YS_ERR_ARG;
  if (!p.assigned) return YS_ERR_STATE;
  cudaError_t e = cudaMemcpyAsync(dst, p.d_mesh, sizeof(float) * (size_t)total, cudaMemcpyDefault, p.stream);
  if (!e) e = cudaStreamSynchronize(p.stream);
  return e ? ys::cuda_fail(e) : YS_OK;
}

ys_status ys_plan_set_profiling(ys_plan* plan, int enable) {
  if (!plan) return YS_ERR_ARG;
  plan->p.profiling = enable != 0;
  return YS_OK;
}

ys_status ys_plan_get_stats(ys_plan* plan, ys_stats* out, int reset) {
  if (!plan || !out) return YS_ERR_ARG;
  Plan& p = plan->p;
  cudaError_t e = p.stream ? cudaStreamSynchronize(p.stream) : cudaDeviceSynchronize();
  if (e) return ys::cuda_fail(e);
  for (auto& ev : p.pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ev.a, ev.b) == cudaSuccess) p.ms[ev.cls] += t;
    p.event_pool.push_back(ev.a);
    p.event_pool.push_back(ev.b);
  }
  p.pending.clear();
  for (int c = 0; c < YS_NUM_KERNEL_CLASSES; ++c) {
    out->launches[c] = p.launches[c];
    out->ms[c] = p.ms[c];
    if (reset) {
      p.launches[c] = 0;
      p.ms[c] = 0.0;
    }
  }
  return YS_OK;
}

}  // extern "C"
