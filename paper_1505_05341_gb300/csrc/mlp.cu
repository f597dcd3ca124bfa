// Learned aliasing / window correction (no counterpart in the paper's equations):
// a 5 -> 64 -> 64 -> 64 -> 3 network with GELU (erf form) on the hidden layers maps
// per-shell features of a coarse-mesh measurement to the residual against a fine
// mesh, (P_l^fine - P_l^coarse) / D with D = P_0 + S/I the coarse monopole before
// shot-noise subtraction.
//
// Weights are kept in bfloat16 for the forward and backward passes (FP32 master copy
// and Adam moments); activations and every accumulation are FP32.  A CTA handles
// MLP_ROWS rows: per-row phases run one row per thread with activations in shared
// memory laid out [feature][row] (odd row stride, so a warp's rows hit distinct
// banks), the weight-gradient contractions run one weight per thread over the CTA's
// rows, and each CTA adds its partial gradient to the global FP32 gradient with
// atomics.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <string>
#include <vector>

#include "ys_internal.h"

namespace ys {
namespace {

constexpr int MLP_ROWS = 64;   // rows (and threads) per CTA
constexpr int RS = MLP_ROWS + 1;  // padded row stride of the [feature][row] buffers
constexpr int H = 64;
constexpr int IN = 5, OUT = 3;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * H, OFF_W4 = OFF_B3 + H, OFF_B4 = OFF_W4 + OUT * H;
constexpr int NP = OFF_B4 + OUT;
static_assert(NP == YS_MLP_PARAMS, "parameter count");

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

struct MlpSmem {
  float w[NP];
  float x[IN * RS];
  float z[3][H * RS];   // pre-activations of the hidden layers (overwritten by deltas)
  float h[3][H * RS];   // post-activations
  float d4[OUT * RS];
};

__device__ __forceinline__ void load_weights(float* w, const __nv_bfloat16* __restrict__ w16) {
  for (int k = threadIdx.x; k < NP; k += blockDim.x) w[k] = __bfloat162float(w16[k]);
}

// One dense layer for this thread's row r: out[o][r] = b[o] + sum_i W[o][i] in[i][r].
__device__ __forceinline__ void dense_row(const float* W, const float* b, const float* in, int nin, float* out,
                                          int nout, int r) {
  for (int o = 0; o < nout; ++o) {
    float acc = b[o];
    const float* wr = W + o * nin;
    for (int i = 0; i < nin; ++i) acc = fmaf(wr[i], in[i * RS + r], acc);
    out[o * RS + r] = acc;
  }
}

// Forward pass of the CTA's rows; keeps z and h for the backward pass.
__device__ __forceinline__ void forward_rows(MlpSmem& s, int rows, float (&y)[OUT]) {
  const int r = threadIdx.x;
  const bool ok = r < rows;
  if (ok) {
    dense_row(s.w + OFF_W1, s.w + OFF_B1, s.x, IN, s.z[0], H, r);
    for (int o = 0; o < H; ++o) s.h[0][o * RS + r] = gelu(s.z[0][o * RS + r]);
    dense_row(s.w + OFF_W2, s.w + OFF_B2, s.h[0], H, s.z[1], H, r);
    for (int o = 0; o < H; ++o) s.h[1][o * RS + r] = gelu(s.z[1][o * RS + r]);
    dense_row(s.w + OFF_W3, s.w + OFF_B3, s.h[1], H, s.z[2], H, r);
    for (int o = 0; o < H; ++o) s.h[2][o * RS + r] = gelu(s.z[2][o * RS + r]);
    for (int o = 0; o < OUT; ++o) {
      float acc = s.w[OFF_B4 + o];
      for (int i = 0; i < H; ++i) acc = fmaf(s.w[OFF_W4 + o * H + i], s.h[2][i * RS + r], acc);
      y[o] = acc;
    }
  }
}

__global__ void __launch_bounds__(MLP_ROWS) k_mlp_forward(const __nv_bfloat16* __restrict__ w16,
                                                          const float* __restrict__ X, int64_t rows,
                                                          float* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char raw[];
  MlpSmem& s = *reinterpret_cast<MlpSmem*>(raw);
  load_weights(s.w, w16);
  const int64_t r0 = (int64_t)blockIdx.x * MLP_ROWS;
  const int nr = rows - r0 < MLP_ROWS ? (int)(rows - r0) : MLP_ROWS;
  for (int k = threadIdx.x; k < IN * MLP_ROWS; k += blockDim.x) {
    const int f = k / MLP_ROWS, r = k % MLP_ROWS;
    s.x[f * RS + r] = r < nr ? X[(r0 + r) * IN + f] : 0.f;
  }
  __syncthreads();
  float y[OUT];
  forward_rows(s, nr, y);
  if ((int)threadIdx.x < nr)
    for (int o = 0; o < OUT; ++o) Y[(r0 + threadIdx.x) * OUT + o] = y[o];
}

// dW[o][i] += sum_r D[o][r] A[i][r] and db[o] += sum_r D[o][r] over the CTA's rows.
__device__ __forceinline__ void weight_grad(const float* D, const float* A, int nout, int nin, int rows,
                                            float* __restrict__ gW, float* __restrict__ gb) {
  for (int k = threadIdx.x; k < nout * nin; k += blockDim.x) {
    const int o = k / nin, i = k % nin;
    float acc = 0.f;
    for (int r = 0; r < rows; ++r) acc = fmaf(D[o * RS + r], A[i * RS + r], acc);
    atomicAdd(&gW[k], acc);
  }
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    float acc = 0.f;
    for (int r = 0; r < rows; ++r) acc += D[o * RS + r];
    atomicAdd(&gb[o], acc);
  }
}

// Delta of a hidden layer for this thread's row: Z[i][r] <- (sum_o W[o][i] D[o][r]) gelu'(Z[i][r]).
__device__ __forceinline__ void back_row(const float* W, const float* D, int nout, float* Z, int nin, int r) {
  for (int i = 0; i < nin; ++i) {
    float acc = 0.f;
    for (int o = 0; o < nout; ++o) acc = fmaf(W[o * nin + i], D[o * RS + r], acc);
    Z[i * RS + r] = acc * gelu_grad(Z[i * RS + r]);
  }
}

// Gradient of loss = sum (y - t)^2 / (rows_total * 3) accumulated into grad; the
// summed squared error goes to sse.
__global__ void __launch_bounds__(MLP_ROWS) k_mlp_backward(const __nv_bfloat16* __restrict__ w16,
                                                           const float* __restrict__ X, const float* __restrict__ T,
                                                           int64_t rows, float* __restrict__ grad,
                                                           double* __restrict__ sse) {
  extern __shared__ __align__(16) unsigned char raw[];
  MlpSmem& s = *reinterpret_cast<MlpSmem*>(raw);
  __shared__ double red[MLP_ROWS / 32];
  load_weights(s.w, w16);
  const int64_t r0 = (int64_t)blockIdx.x * MLP_ROWS;
  const int nr = rows - r0 < MLP_ROWS ? (int)(rows - r0) : MLP_ROWS;
  for (int k = threadIdx.x; k < IN * MLP_ROWS; k += blockDim.x) {
    const int f = k / MLP_ROWS, r = k % MLP_ROWS;
    s.x[f * RS + r] = r < nr ? X[(r0 + r) * IN + f] : 0.f;
  }
  __syncthreads();
  float y[OUT];
  forward_rows(s, nr, y);
  const int r = threadIdx.x;
  const float scale = 2.f / (float)(rows * OUT);
  double e2 = 0.0;
  for (int o = 0; o < OUT; ++o) {
    float d = 0.f;
    if (r < nr) {
      const float diff = y[o] - T[(r0 + r) * OUT + o];
      e2 += (double)diff * diff;
      d = scale * diff;
    }
    s.d4[o * RS + r] = d;
  }
  // rows beyond nr contribute zero deltas; their activations are zeroed too
  if (r >= nr)
    for (int l = 0; l < 3; ++l)
      for (int i = 0; i < H; ++i) s.h[l][i * RS + r] = 0.f;
  __syncthreads();
  weight_grad(s.d4, s.h[2], OUT, H, MLP_ROWS, grad + OFF_W4, grad + OFF_B4);
  __syncthreads();
  if (r < nr) back_row(s.w + OFF_W4, s.d4, OUT, s.z[2], H, r);
  else for (int i = 0; i < H; ++i) s.z[2][i * RS + r] = 0.f;
  __syncthreads();
  weight_grad(s.z[2], s.h[1], H, H, MLP_ROWS, grad + OFF_W3, grad + OFF_B3);
  __syncthreads();
  if (r < nr) back_row(s.w + OFF_W3, s.z[2], H, s.z[1], H, r);
  else for (int i = 0; i < H; ++i) s.z[1][i * RS + r] = 0.f;
  __syncthreads();
  weight_grad(s.z[1], s.h[0], H, H, MLP_ROWS, grad + OFF_W2, grad + OFF_B2);
  __syncthreads();
  if (r < nr) back_row(s.w + OFF_W2, s.z[1], H, s.z[0], H, r);
  else for (int i = 0; i < H; ++i) s.z[0][i * RS + r] = 0.f;
  __syncthreads();
  weight_grad(s.z[0], s.x, H, IN, MLP_ROWS, grad + OFF_W1, grad + OFF_B1);
  // squared error
  for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < MLP_ROWS / 32; ++k) t += red[k];
    atomicAdd(sse, t);
  }
}

// Adam on the FP32 master weights, refresh of the bfloat16 copy, gradient reset.
__global__ void k_mlp_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ w16, float* __restrict__ grad,
                           float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NP) return;
  const float g = grad[k];
  const float mk = b1 * m[k] + (1.f - b1) * g;
  const float vk = b2 * v[k] + (1.f - b2) * g * g;
  m[k] = mk;
  v[k] = vk;
  const float wk = w[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
  w[k] = wk;
  w16[k] = __float2bfloat16_rn(wk);
  grad[k] = 0.f;
}

// Per-shell features of result rows (layout of ys_measure_multipoles_async) and,
// when fine rows are given, the targets.  A shell enters when it has modes, finite
// multipoles and D > 0.  Rows are appended in an order set by atomics; src[] maps
// each row back to (catalogue * n_bins + shell).
__global__ void k_mlp_features(const double* __restrict__ rows, const double* __restrict__ fine, int n_cat,
                               int64_t stride, int n_bins, double k_nyq, float* __restrict__ X,
                               float* __restrict__ T, int* __restrict__ src, int* __restrict__ count) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_cat * n_bins) return;
  const int c = idx / n_bins, b = idx % n_bins;
  const double* row = rows + (size_t)c * stride;
  const double nm = row[n_bins + b];
  const double p0 = row[2 * n_bins + b], p2 = row[3 * n_bins + b], p4 = row[4 * n_bins + b];
  const double psn = row[5 * n_bins + 2];
  const double D = p0 + psn;
  if (!(nm > 0) || !isfinite(p0) || !isfinite(p2) || !isfinite(p4) || !(psn > 0) || !(D > 0)) return;
  double t0 = 0, t2 = 0, t4 = 0;
  if (fine) {
    const double* fr = fine + (size_t)c * stride;
    const double f0 = fr[2 * n_bins + b], f2 = fr[3 * n_bins + b], f4 = fr[4 * n_bins + b];
    if (!isfinite(f0) || !isfinite(f2) || !isfinite(f4)) return;
    t0 = (f0 - p0) / D;
    t2 = (f2 - p2) / D;
    t4 = (f4 - p4) / D;
  }
  const int slot = atomicAdd(count, 1);
  float* x = X + (size_t)slot * IN;
  x[0] = (float)(row[b] / k_nyq);
  x[1] = (float)log(D / psn);
  x[2] = (float)(p2 / D);
  x[3] = (float)(p4 / D);
  x[4] = (float)(psn / D);
  if (T) {
    T[(size_t)slot * OUT + 0] = (float)t0;
    T[(size_t)slot * OUT + 1] = (float)t2;
    T[(size_t)slot * OUT + 2] = (float)t4;
  }
  src[slot] = idx;
}

// P_l <- P_l + D y_l for each featured shell (in place on out, which already holds
// a copy of rows).
__global__ void k_mlp_apply(const double* __restrict__ rows, int64_t stride, int n_bins, const float* __restrict__ Y,
                            const int* __restrict__ src, const int* __restrict__ count, double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *count) return;
  const int idx = src[k];
  const int c = idx / n_bins, b = idx % n_bins;
  const double* row = rows + (size_t)c * stride;
  const double D = row[2 * n_bins + b] + row[5 * n_bins + 2];
  for (int l = 0; l < OUT; ++l)
    out[(size_t)c * stride + (2 + l) * n_bins + b] = row[(2 + l) * n_bins + b] + D * (double)Y[(size_t)k * OUT + l];
}

}  // namespace
}  // namespace ys

struct ys_mlp_s {
  float* w = nullptr;            // FP32 master weights
  __nv_bfloat16* w16 = nullptr;  // bfloat16 copy used by the kernels
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  double* sse = nullptr;
  float* fx = nullptr;           // feature scratch for ys_mlp_correct
  float* fy = nullptr;
  int* fsrc = nullptr;
  int* fcount = nullptr;
  int64_t fcap = 0;
  int64_t t = 0;                 // Adam steps taken
};

namespace {

size_t smem_bytes() { return sizeof(ys::MlpSmem); }

ys_status fail(cudaError_t e) {
  ys::g_last_cuda_error = cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? YS_ERR_OOM : YS_ERR_CUDA;
}

void free_mlp(ys_mlp* m) {
  for (void* p : {(void*)m->w, (void*)m->w16, (void*)m->grad, (void*)m->m, (void*)m->v, (void*)m->sse,
                  (void*)m->fx, (void*)m->fy, (void*)m->fsrc, (void*)m->fcount})
    if (p) cudaFree(p);
  delete m;
}

cudaError_t set_attrs() {
  cudaError_t e = cudaFuncSetAttribute(ys::k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
  if (!e) e = cudaFuncSetAttribute(ys::k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
  return e;
}

}  // namespace

extern "C" {

ys_status ys_mlp_create(const float* h_params, ys_mlp** out) {
  if (!h_params || !out) return YS_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    ys::g_last_cuda_error = "no CUDA device";
    return YS_ERR_CUDA;
  }
  ys_mlp* m = new (std::nothrow) ys_mlp;
  if (!m) return YS_ERR_OOM;
  cudaError_t e;
  const size_t n = ys::NP;
  if ((e = cudaMalloc(&m->w, n * 4)) || (e = cudaMalloc(&m->w16, n * 2)) || (e = cudaMalloc(&m->grad, n * 4)) ||
      (e = cudaMalloc(&m->m, n * 4)) || (e = cudaMalloc(&m->v, n * 4)) || (e = cudaMalloc(&m->sse, 8)) ||
      (e = cudaMalloc(&m->fcount, 4))) {
    free_mlp(m);
    return fail(e);
  }
  std::vector<__nv_bfloat16> h16(n);
  for (size_t k = 0; k < n; ++k) h16[k] = __float2bfloat16_rn(h_params[k]);
  if ((e = cudaMemcpy(m->w, h_params, n * 4, cudaMemcpyHostToDevice)) ||
      (e = cudaMemcpy(m->w16, h16.data(), n * 2, cudaMemcpyHostToDevice)) || (e = cudaMemset(m->grad, 0, n * 4)) ||
      (e = cudaMemset(m->m, 0, n * 4)) || (e = cudaMemset(m->v, 0, n * 4)) || (e = set_attrs())) {
    free_mlp(m);
    return fail(e);
  }
  *out = m;
  return YS_OK;
}

ys_status ys_mlp_get_state(ys_mlp* m, float* h_params, float* h_m, float* h_v, int64_t* h_step) {
  if (!m) return YS_ERR_ARG;
  cudaError_t e = cudaDeviceSynchronize();
  if (!e && h_params) e = cudaMemcpy(h_params, m->w, ys::NP * 4, cudaMemcpyDeviceToHost);
  if (!e && h_m) e = cudaMemcpy(h_m, m->m, ys::NP * 4, cudaMemcpyDeviceToHost);
  if (!e && h_v) e = cudaMemcpy(h_v, m->v, ys::NP * 4, cudaMemcpyDeviceToHost);
  if (e) return fail(e);
  if (h_step) *h_step = m->t;
  return YS_OK;
}

ys_status ys_mlp_set_state(ys_mlp* m, const float* h_params, const float* h_m, const float* h_v, int64_t step) {
  if (!m || !h_params || step < 0) return YS_ERR_ARG;
  const size_t n = ys::NP;
  std::vector<__nv_bfloat16> h16(n);
  for (size_t k = 0; k < n; ++k) h16[k] = __float2bfloat16_rn(h_params[k]);
  cudaError_t e = cudaDeviceSynchronize();
  if (!e) e = cudaMemcpy(m->w, h_params, n * 4, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(m->w16, h16.data(), n * 2, cudaMemcpyHostToDevice);
  if (!e) e = h_m ? cudaMemcpy(m->m, h_m, n * 4, cudaMemcpyHostToDevice) : cudaMemset(m->m, 0, n * 4);
  if (!e) e = h_v ? cudaMemcpy(m->v, h_v, n * 4, cudaMemcpyHostToDevice) : cudaMemset(m->v, 0, n * 4);
  if (e) return fail(e);
  m->t = step;
  return YS_OK;
}

ys_status ys_mlp_forward(ys_mlp* m, const float* d_x, int64_t rows, float* d_y, void* stream) {
  if (!m || rows < 0 || (rows > 0 && (!d_x || !d_y))) return YS_ERR_ARG;
  if (rows == 0) return YS_OK;
  const int64_t blocks = (rows + ys::MLP_ROWS - 1) / ys::MLP_ROWS;
  ys::k_mlp_forward<<<(unsigned)blocks, ys::MLP_ROWS, smem_bytes(), static_cast<cudaStream_t>(stream)>>>(
      m->w16, d_x, rows, d_y);
  cudaError_t e = cudaGetLastError();
  return e ? fail(e) : YS_OK;
}

ys_status ys_mlp_gradient(ys_mlp* m, const float* d_x, const float* d_t, int64_t rows, float* d_grad,
                          double* d_loss, void* stream) {
  if (!m || rows <= 0 || !d_x || !d_t) return YS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = cudaMemsetAsync(m->grad, 0, ys::NP * 4, st)) || (e = cudaMemsetAsync(m->sse, 0, 8, st))) return fail(e);
  const int64_t blocks = (rows + ys::MLP_ROWS - 1) / ys::MLP_ROWS;
  ys::k_mlp_backward<<<(unsigned)blocks, ys::MLP_ROWS, smem_bytes(), st>>>(m->w16, d_x, d_t, rows, m->grad, m->sse);
  if ((e = cudaGetLastError())) return fail(e);
  if (d_grad && (e = cudaMemcpyAsync(d_grad, m->grad, ys::NP * 4, cudaMemcpyDeviceToDevice, st))) return fail(e);
  if (d_loss && (e = cudaMemcpyAsync(d_loss, m->sse, 8, cudaMemcpyDeviceToDevice, st))) return fail(e);
  return YS_OK;
}

ys_status ys_mlp_train_step(ys_mlp* m, const float* d_x, const float* d_t, int64_t rows, float lr, double* d_sse,
                            void* stream) {
  ys_status s = ys_mlp_gradient(m, d_x, d_t, rows, nullptr, d_sse, stream);
  if (s != YS_OK) return s;
  m->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)m->t), c2 = 1.f - powf(b2, (float)m->t);
  ys::k_mlp_adam<<<(ys::NP + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(m->w, m->w16, m->grad, m->m,
                                                                                       m->v, lr, b1, b2, 1e-8f, c1, c2);
  cudaError_t e = cudaGetLastError();
  return e ? fail(e) : YS_OK;
}

ys_status ys_mlp_features(const double* d_rows, const double* d_fine_rows, int32_t n_cat, int64_t stride,
                          int32_t n_bins, double k_nyq, float* d_x, float* d_t, int32_t* d_src, int32_t* d_count,
                          void* stream) {
  if (!d_rows || n_cat <= 0 || n_bins <= 0 || stride < 5 * (int64_t)n_bins + 5 || !(k_nyq > 0) || !d_x || !d_src ||
      !d_count || (d_fine_rows && !d_t))
    return YS_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(d_count, 0, 4, st);
  if (e) return fail(e);
  const int total = n_cat * n_bins;
  ys::k_mlp_features<<<(total + 255) / 256, 256, 0, st>>>(d_rows, d_fine_rows, n_cat, stride, n_bins, k_nyq, d_x,
                                                          d_fine_rows ? d_t : nullptr, d_src, d_count);
  e = cudaGetLastError();
  return e ? fail(e) : YS_OK;
}

ys_status ys_mlp_correct(ys_mlp* m, const double* d_rows, int32_t n_cat, int64_t stride, int32_t n_bins,
                         double k_nyq, double* d_out, void* stream) {
  if (!m || !d_rows || !d_out || n_cat <= 0 || n_bins <= 0 || stride < 5 * (int64_t)n_bins + 5) return YS_ERR_ARG;
  if (d_out != d_rows && d_out < d_rows + (size_t)n_cat * stride && d_rows < d_out + (size_t)n_cat * stride)
    return YS_ERR_ARG;  // partial overlap
  const int64_t need = (int64_t)n_cat * n_bins;
  cudaError_t e;
  if (need > m->fcap) {
    if (m->fx) cudaFree(m->fx);
    if (m->fy) cudaFree(m->fy);
    if (m->fsrc) cudaFree(m->fsrc);
    m->fx = nullptr;
    m->fy = nullptr;
    m->fsrc = nullptr;
    if ((e = cudaMalloc(&m->fx, need * 5 * 4)) || (e = cudaMalloc(&m->fy, need * 3 * 4)) ||
        (e = cudaMalloc(&m->fsrc, need * 4)))
      return fail(e);
    m->fcap = need;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ys_status s = ys_mlp_features(d_rows, nullptr, n_cat, stride, n_bins, k_nyq, m->fx, nullptr, m->fsrc, m->fcount,
                                stream);
  if (s != YS_OK) return s;
  // all n_cat * n_bins slots are evaluated; slots past *count hold no row and are not used
  s = ys_mlp_forward(m, m->fx, need, m->fy, stream);
  if (s != YS_OK) return s;
  if (d_out != d_rows &&
      (e = cudaMemcpyAsync(d_out, d_rows, sizeof(double) * (size_t)(n_cat * stride), cudaMemcpyDeviceToDevice, st)))
    return fail(e);
  ys::k_mlp_apply<<<(unsigned)((need + 255) / 256), 256, 0, st>>>(d_rows, stride, n_bins, m->fy, m->fsrc, m->fcount,
                                                                 d_out);
  e = cudaGetLastError();
  return e ? fail(e) : YS_OK;
}

ys_status ys_mlp_destroy(ys_mlp* m) {
  if (!m) return YS_OK;
  cudaDeviceSynchronize();
  free_mlp(m);
  return YS_OK;
}

}  // extern "C"
