// Internal plan state and kernel entry points of the ystat library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "ystat.h"  // include/ (on the -I path)

namespace ys {

// Catalogue sums accumulated in FP64 (Eq. 1 and Eq. 3):
enum SumSlot {
  SUM_WG = 0,    // sum_gal w
  SUM_WG2 = 1,   // sum_gal w^2
  SUM_WR = 2,    // sum_ran w
  SUM_WR2 = 3,   // sum_ran w^2
  SUM_WR2N = 4,  // sum_ran w^2 nbar
  SUM_BAD = 5,   // particles outside the box
  SUM_TIMEOUT = 6,   // set when a bounded device-side wait ran out
  SUM_COUNT = 8
};

// Tile of the scatter: TX x TY x TZ mesh nodes per CTA (capped at N per axis); the
// default and the shapes the autotuner tries (each divides every supported N once
// capped; shared memory = meshes x nodes x 4 bytes).
constexpr int TILE_X = 16, TILE_Y = 16, TILE_Z = 16;

// Most catalogues of one configuration measured in one set of spectral launches.
constexpr int YZ_MAX_LANES = 8;

// Pencils per CTA of the x stage (its FFT tile): the default for mesh size n and the
// alternative the autotuner also times.  Both are powers of two; the plan pads its
// pencil list to a multiple of the larger.
__host__ __device__ constexpr int k3_pencils(int n) { return n <= 32 ? 32 : (n >= 512 ? 4 : 8); }
__host__ __device__ constexpr int k3_pencils_alt(int n) {
  return n <= 32 ? 16 : (n >= 1024 ? 2 : (n >= 512 ? 8 : 4));
}
constexpr int kTileCandidates[5][3] = {{16, 16, 32}, {8, 16, 32}, {16, 16, 16}, {32, 16, 32}, {8, 8, 32}};

struct Geom {
  int n;            // mesh side N
  float inv_h;      // 1 / H
  float bmin[3];    // box_min (float) for the first guess of the cell index
  int tiles[3];     // tiles per axis
  int tdim[3];      // tile extent per axis
};

struct Plan {
  ys_config cfg;
  cudaStream_t stream = nullptr;
  int n = 0, m = 1, ell = 0, kind = 2;
  int nb = 1, ng = 1;            // basis fields / k_x-power groups
  int row_len = 0;               // doubles in a result row (result_row_len)
  double H = 0, kf = 0;
  Geom geom{};
  int ntiles = 0;
  // pencils (k_y, k_z) kept for the x transform: k_y^2 + k_z^2 < n2_hi
  int n2_hi = 0, nzc = 0, np = 0;
  int np_pad = 0;                // np rounded up to whole x-stage pencil blocks (of either size)
  int x_pencils = 0;             // pencils per x-stage CTA in use (k3_pencils or k3_pencils_alt)
  int ring_slots = 1;            // S: planes held by the y,z-stage ring
  int ring_lead = 1;             // D: column items trail row items by D planes
  int ring_lead_pct = 100;       // D relative to the work-balanced estimate (tuned)
  int ring_slots_cap = 0;        // ring slots allocated
  int yz_grid = 1;               // CTAs of the persistent y,z kernel
  int yz_grid_max = 1;           // resident CTAs of that kernel (upper bound for tuning)
  long long yz_wait_ns = 1000000000LL;  // bound of each y,z-stage wait (ns)
  int fault_skip_plane = -1;     // test hook: plane whose row items withhold their completion
  int ntiles_max = 0;            // tile-counter capacity over the scatter tile candidates
  bool direct_assign = false;    // assignment by global reductions into an L2-resident mesh
  bool direct_ok = false;        // the mesh set is small enough for it (m N^3 floats <= 64 MB)
  // device tables
  float2* d_tw = nullptr;        // [n] exp(-2 pi i j / n)
  float2* d_nodes = nullptr;     // [3][n + 3] node positions (hi, lo), index offset 1
  float* d_rel = nullptr;        // [m][3][n] node - observer (float)
  float* d_invw = nullptr;       // [n] per-axis 1 / sinc^p by FFT index (1 if !compensate)
  float2* d_phase = nullptr;     // [n] per-axis exp(-i pi m / n) by FFT index
  int* d_col_off = nullptr;      // [nzc + 1] first pencil of each k_z column
  short2* d_pencil = nullptr;    // [np] (k_y signed, k_z)
  short* d_lut = nullptr;        // [n2_hi] shell index of |m|^2, -1 = not used
  double* d_shell = nullptr;     // [2][n_bins] mode count and sum |k| (host-built)
  // buffers
  float* d_mesh = nullptr;       // [m][n][n][n]
  float2* d_z = nullptr;         // [S][nb][nzc][n] y,z-stage ring of z-transformed planes
  int* d_sync = nullptr;         // [2 m n + 2] per-plane counters, ticket, error flag
  float2* d_g = nullptr;         // [m][ng][n][np_pad] grouped y,z transforms
  CUtensorMap gmap;              // 2D tensor map of d_g for the x-stage TMA loads
  double* d_acc = nullptr;       // [4][n_bins] shell sums (slot 3 for l_max = 6)
  double* d_sums = nullptr;      // [SUM_COUNT]
  double* d_result = nullptr;    // [5 n_bins + 3]
  unsigned* d_tile_count = nullptr;  // [ntiles]
  unsigned* d_tile_off = nullptr;    // [ntiles + 1]
  unsigned* d_tile_cur = nullptr;    // [ntiles]
  float4* d_rec = nullptr;       // [rec_cap] (x, y, z, signed weight) per (particle, tile)
  // shared randoms (ys_randoms_cache): sum_ran w W per mesh node, and its FP64 sums
  float* d_rmesh = nullptr;      // [m][n][n][n]
  double* d_rsums = nullptr;     // [3] sum w, sum w^2, sum w^2 nbar
  bool randoms_cached = false;
  int64_t rec_cap = 0;
  int64_t part_cap = 0;
  // host staging for ys_estimate_host
  float* d_stage = nullptr;
  int64_t stage_cap = 0;
  std::vector<double> h_result;
  size_t device_bytes = 0;
  bool assigned = false;
  // CUDA graph of the measurement sequence (all pointers are plan-owned)
  cudaStream_t cap_stream = nullptr;
  // ys_estimate_host: extra streams that carry part of the host -> device copies in
  // parallel with the plan's stream, and the events that fork and join them
  static constexpr int kCopyStreams = 3;
  cudaStream_t copy_stream[kCopyStreams] = {};
  cudaEvent_t copy_event[kCopyStreams + 1] = {};
  cudaGraphExec_t measure_exec = nullptr;
  int64_t measure_launches[YS_NUM_KERNEL_CLASSES] = {};
  // statistics and optional event profiling
  bool profiling = false;
  bool capturing = false;
  int64_t launches[YS_NUM_KERNEL_CLASSES] = {};
  double ms[YS_NUM_KERNEL_CLASSES] = {};
  struct EvPair { cudaEvent_t a, b; int cls; };
  std::vector<EvPair> pending;
  std::vector<cudaEvent_t> event_pool;
};

// Brackets one kernel launch: counts it and, when profiling, records events.
struct LaunchScope {
  Plan& p;
  int cls;
  cudaEvent_t a = nullptr, b = nullptr;
  LaunchScope(Plan& plan, int c);
  ~LaunchScope();
};

// Kernel launchers (return cudaError_t of the launch).
// rmesh / rsums: shared randoms (ys_assign_cached); nullptr for a plain assignment.
cudaError_t launch_assign(Plan& p, const ys_catalog& gal, const ys_catalog& ran, const float* rmesh = nullptr,
                          const double* rsums = nullptr);
// FP64 sum w, sum w^2, sum w^2 nbar of a random catalogue into out[3].
cudaError_t launch_random_sums(Plan& p, const ys_catalog& ran, double* out);
// Scatter tile shape (nodes per axis, capped at N); updates geom and ntiles.
void set_tiles(Plan& p, int tx, int ty, int tz);
// Pencils per x-stage CTA (k3_pencils or k3_pencils_alt of N): re-encodes the tensor
// map of the grouped transforms for that box and drops the captured graph.
ys_status set_x_pencils(Plan& p, int pencils);
// y,z grid size; updates the ring lead D and slots S (S never exceeds the allocation).
void set_yz_grid(Plan& p, int grid, int lead_pct = 0);
constexpr int kRingLeadPctMax = 200;

// Rows (x values) per TMA box of the x stage: a divisor of N no larger than the
// 256-element limit of a box dimension (N = 384 -> 192).
__host__ __device__ constexpr int x_box_rows(int n) {
  return n <= 256 ? n : (n % 256 == 0 ? 256 : (n % 192 == 0 ? 192 : 128));
}
ys_status ensure_particles(Plan& p, int64_t total);
// Doubles in a result row: 5 n_bins + 5, plus n_bins of P_6 for l_max = 6.
inline int result_row_len(int nbins, int ell) { return 5 * nbins + 5 + (ell >= 6 ? nbins : 0); }
extern thread_local std::string g_last_cuda_error;
cudaError_t launch_measure(Plan& p);
// The measurement of W <= 8 plans of one configuration (each already assigned) in one
// y,z launch, one x-stage launch and one finalize launch; lane l's result row goes to
// rows[l].  Queued on lanes[0]'s stream.
cudaError_t launch_measure_lanes(Plan* const* lanes, int W, double* const* rows);
ys_status assign_noalloc(Plan& p, const ys_catalog& gal, const ys_catalog& ran, std::string& why);

}  // namespace ys

struct ys_plan_s {
  ys::Plan p;
};
