// ys_assign_noalloc: the mesh-assignment step with its scratch (per-tile counters
// and the per-tile particle records of the counting sort) in a fixed, file-scope
// device array instead of plan-owned cudaMalloc buffers.
//
// ys_assign sizes its record buffers to the catalogue and grows them with
// cudaMalloc when a larger catalogue arrives.  Some callers cannot allocate device
// memory at that point -- for example code running under a memory pool that must not
// grow, or an embedding framework that forbids the library from calling cudaMalloc
// after set-up.  This entry point never allocates: it borrows a static array that
// every GPU loading the library holds for the life of the process, and refuses
// catalogues that do not fit in it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "ys_internal.h"

namespace ys {
namespace {

constexpr size_t NOALLOC_BYTES = (size_t)YS_NOALLOC_SCRATCH_BYTES;

// The shared scratch.  In host code this name is only a stand-in for the device
// symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void* g_scratch_ptr[MAX_DEVICES] = {};
void* g_scratch_ctx[MAX_DEVICES] = {};  // context the address was looked up in

// The current CUDA context (driver handle), through the runtime's driver entry point.
cudaError_t current_context(void** ctx) {
  using GetCurrent = int (*)(void**);
  static GetCurrent fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (!f || q != cudaDriverEntryPointSuccess) return cudaErrorNotSupported;
    fn = reinterpret_cast<GetCurrent>(f);
  }
  return fn(ctx) == 0 ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of the scratch on the current device, looked up once per device
// with that device current, and again if the device's context has changed since
// (after cudaDeviceReset the module, and the array with it, is loaded anew).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  // (a null context here -- none made current yet -- only costs one more lookup later)
  void* ctx = nullptr;
  if ((e = current_context(&ctx)) != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = ptr;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

ys_status assign_noalloc(Plan& p, const ys_catalog& gal, const ys_catalog& ran, std::string& why) {
  int factor = 1;
  for (int a = 0; a < 3; ++a) factor *= p.geom.tiles[a] > 1 ? 2 : 1;
  const size_t nt = (size_t)p.ntiles;
  const size_t records = (size_t)(gal.n + ran.n) * factor;
  // Layout: tile counts | tile offsets | tile cursors | records (float4)
  const size_t off_off = align256(nt * sizeof(unsigned));
  const size_t off_cur = off_off + align256((nt + 1) * sizeof(unsigned));
  const size_t off_rec = off_cur + align256(nt * sizeof(unsigned));
  const size_t need = off_rec + records * sizeof(float4);
  if (need > NOALLOC_BYTES) {
    why = "catalogue too large for the no-allocation scratch: " + std::to_string(gal.n + ran.n) +
          " particles need " + std::to_string(need) + " bytes (up to " + std::to_string(factor) +
          " tile records each), the limit is " + std::to_string(NOALLOC_BYTES) + " bytes";
    return YS_ERR_UNSUPPORTED;
  }
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) {
    why = cudaGetErrorString(e);
    return YS_ERR_CUDA;
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  // Point the plan's sort buffers at the scratch for this call only; the launch
  // sequence is the one ys_assign uses (it zeroes the tile counters and the sums).
  unsigned* s_count = p.d_tile_count;
  unsigned* s_off = p.d_tile_off;
  unsigned* s_cur = p.d_tile_cur;
  float4* s_rec = p.d_rec;
  p.d_tile_count = reinterpret_cast<unsigned*>(b);
  p.d_tile_off = reinterpret_cast<unsigned*>(b + off_off);
  p.d_tile_cur = reinterpret_cast<unsigned*>(b + off_cur);
  p.d_rec = reinterpret_cast<float4*>(b + off_rec);
  e = launch_assign(p, gal, ran);
  p.d_tile_count = s_count;
  p.d_tile_off = s_off;
  p.d_tile_cur = s_cur;
  p.d_rec = s_rec;
  if (e != cudaSuccess) {
    why = cudaGetErrorString(e);
    return YS_ERR_CUDA;
  }
  p.assigned = true;
  return YS_OK;
}

}  // namespace ys
