// Learned flow initializer: inference and training kernels (device code of
// the network in initnet_dev.cuh).
//
//  pack     FP32 master parameters -> BF16 [N][K] matrices + FP32 biases
//  extract  network inputs of keypoints from two pyramids
//  forward  persistent CTAs of 128 threads over rounds of 32 samples, layer
//           by layer on the tcgen05 tensor cores (initnet_tc.cuh: BF16
//           operands in shared memory, FP32 accumulators in tensor memory)
//  train    the forward pass of one sample per warp (same layers, BF16
//           activations), then the backward pass in FP32 per warp, with
//           the weight gradients summed in shared memory per CTA and added to
//           the global gradient once per CTA
//  adam     Adam update of the master parameters
#include <math.h>

#include "initnet_dev.cuh"
#include "initnet_tc.cuh"

namespace vio {
namespace {

using namespace net;

__global__ void pack_kernel(const float* __restrict__ m, uint16_t* __restrict__ w,
                            float* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N_BF16) {
    float v = 0.f;
    if (i < OFF_W2) {                     // w1: [32][48], taps 36..47 zero
      const int n = i / K1, k = i % K1;
      if (k < 36) v = m[M_W1 + n * 36 + k];
    } else if (i < OFF_W3) {
      v = m[M_W2 + (i - OFF_W2)];
    } else if (i < OFF_W4) {
      v = m[M_W3 + (i - OFF_W3)];
    } else if (i < OFF_W5) {
      v = m[M_W4 + (i - OFF_W4)];
    } else {                              // w5: [8][64], rows 3..7 zero
      const int n = (i - OFF_W5) / K5, k = (i - OFF_W5) % K5;
      if (n < 3) v = m[M_W5 + n * K5 + k];
    }
    w[i] = f2bf(v);
  }
  if (i < N_BIAS) {
    float v = 0.f;
    if (i < OFF_B2) v = m[M_B1 + i];
    else if (i < OFF_B3) v = m[M_B2 + i - OFF_B2];
    else if (i < OFF_B4) v = m[M_B3 + i - OFF_B3];
    else if (i < OFF_B5) v = m[M_B4 + i - OFF_B4];
    else if (i < OFF_B5 + 3) v = m[M_B5 + i - OFF_B5];
    b[i] = v;
  }
}

struct ExtractArgs {
  Geom g;
  Batch src, dst;
  const float* pts;
  const int32_t* count;
  int capacity, la, lb;
  uint16_t* x;   // [n][4][16][16] bf16
};

__global__ void extract_kernel(ExtractArgs a) {
  __shared__ __align__(16) uint8_t smem[4][WARP_SMEM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long wid = (long long)blockIdx.x * 4 + warp;
  const long long total = (long long)a.capacity * a.src.n;
  if (wid >= total) return;
  const int img = (int)(wid / a.capacity);
  const int k = (int)(wid - (long long)img * a.capacity);
  const int n = a.count ? min(a.count[img], a.capacity) : a.capacity;
  uint16_t* out = a.x + wid * 1024;
  if (k >= n) {
    for (int e = lane; e < 1024; e += 32) out[e] = 0;
    return;
  }
  uint8_t* ws = smem[warp];
  extract_warp(a.g, a.src, img, a.dst, img, a.pts[2 * wid], a.pts[2 * wid + 1], a.la, a.lb, ws,
               lane);
  const uint16_t* xb = reinterpret_cast<const uint16_t*>(ws + S_X);
  for (int e = lane; e < 1024; e += 32) {
    const int ch = e >> 8, r = (e >> 4) & 15, c = e & 15;
    out[e] = xb[ch * XP * XP + (r + 1) * XP + (c + 1)];
  }
}

// copy an unbordered [4][16][16] input into the warp's bordered buffer
__device__ __forceinline__ void load_input(const uint16_t* __restrict__ x, uint8_t* ws,
                                           int lane) {
  uint16_t* xb = reinterpret_cast<uint16_t*>(ws + S_X);
  for (int e = lane; e < 1024; e += 32) {
    const int ch = e >> 8, r = (e >> 4) & 15, c = e & 15;
    xb[ch * XP * XP + (r + 1) * XP + (c + 1)] = x[e];
  }
  __syncwarp();
}

// Status word of the tensor-core forward passes (VIO_ERR_TIMEOUT when one
// gave up waiting for an MMA completion).
__device__ int32_t g_net_fault;

// Inference over n inputs ([n][4][16][16] BF16): persistent CTAs over rounds
// of 32 samples.
__global__ void __launch_bounds__(ntc::THREADS, 1) forward_tc_kernel(
    const void* __restrict__ packed_w, const uint16_t* __restrict__ x, int n,
    float* __restrict__ out, int32_t* fault) {
  extern __shared__ __align__(16) uint8_t sm[];
  const ntc::XSource src{x, n, out};
  ntc::run(src, packed_w, sm, fault);
}

constexpr int TRAIN_WARPS = 4;
// per-warp FP32 backward scratch: da4[64], da3[128], da2[512], da1[2048]
constexpr int BW_FLOATS = 64 + 128 + 512 + 2048;

__device__ __forceinline__ float wgt(const uint16_t* W, int K, int n, int k) {
  return bf2f(W[n * K + k]);
}

__global__ void __launch_bounds__(TRAIN_WARPS * 32) train_kernel(
    const void* __restrict__ packed_w, const uint16_t* __restrict__ x,
    const float* __restrict__ flow, const int32_t* __restrict__ index, int n, float grad_scale,
    float radius, float* __restrict__ grad, float* __restrict__ loss_sum) {
  extern __shared__ __align__(16) uint8_t dsm[];
  float* gacc = reinterpret_cast<float*>(dsm);                       // N_MASTER
  uint8_t* wsm = dsm + ((N_MASTER * 4 + 127) & ~127);               // TRAIN_WARPS x WARP_SMEM
  float* bsm = reinterpret_cast<float*>(wsm + TRAIN_WARPS * WARP_SMEM);  // TRAIN_WARPS x BW
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < N_MASTER; i += blockDim.x) gacc[i] = 0.f;
  uint8_t* ws = wsm + warp * WARP_SMEM;
  float* bw = bsm + warp * BW_FLOATS;
  float* da4 = bw;
  float* da3 = bw + 64;
  float* da2 = bw + 192;
  float* da1 = bw + 704;
  clear_warp_smem(ws, lane);
  __syncthreads();
  const Packed P = packed(packed_w);
  const uint16_t* xb = reinterpret_cast<const uint16_t*>(ws + S_X);
  const uint16_t* h1 = reinterpret_cast<const uint16_t*>(ws + S_H1);
  const uint16_t* h2 = reinterpret_cast<const uint16_t*>(ws + S_H2);
  const uint16_t* h3 = reinterpret_cast<const uint16_t*>(ws + S_H3);
  const uint16_t* h4 = reinterpret_cast<const uint16_t*>(ws + S_H4);
  float lsum = 0.f;
  for (long long sidx = (long long)blockIdx.x * TRAIN_WARPS + warp; sidx < n;
       sidx += (long long)gridDim.x * TRAIN_WARPS) {
    const long long sample = index ? index[sidx] : sidx;
    load_input(x + sample * 1024, ws, lane);
    float o[3];
    forward_warp(P, ws, lane, o);
    __syncwarp();
    // loss and dL/do (the label carries no gradient)
    const float fx = flow[2 * sample], fy = flow[2 * sample + 1];
    const float t0 = fx / kScale, t1 = fy / kScale;
    const float y = hypotf(o[0] * kScale - fx, o[1] * kScale - fy) < radius ? 1.f : 0.f;
    const float sg = 1.f / (1.f + expf(-o[2]));
    const float loss = (o[0] - t0) * (o[0] - t0) + (o[1] - t1) * (o[1] - t1) -
                       (y * logf(sg + 1e-12f) + (1.f - y) * logf(1.f - sg + 1e-12f));
    lsum += loss;
    const float d0 = grad_scale * 2.f * (o[0] - t0);
    const float d1 = grad_scale * 2.f * (o[1] - t1);
    const float d2 = grad_scale * (sg - y);
    // fc2
    for (int k = lane; k < 64; k += 32) {
      const float hk = bf2f(h4[k]);
      atomicAdd(&gacc[M_W5 + 0 * 64 + k], d0 * hk);
      atomicAdd(&gacc[M_W5 + 1 * 64 + k], d1 * hk);
      atomicAdd(&gacc[M_W5 + 2 * 64 + k], d2 * hk);
      const float dh = wgt(P.w + OFF_W5, K5, 0, k) * d0 + wgt(P.w + OFF_W5, K5, 1, k) * d1 +
                       wgt(P.w + OFF_W5, K5, 2, k) * d2;
      da4[k] = hk > 0.f ? dh : 0.f;
    }
    if (lane == 0) {
      atomicAdd(&gacc[M_B5 + 0], d0);
      atomicAdd(&gacc[M_B5 + 1], d1);
      atomicAdd(&gacc[M_B5 + 2], d2);
    }
    __syncwarp();
    // fc1: dW4 = da4 (x) h3, dh3 = W4^T da4
    for (int e = lane; e < 64 * 128; e += 32) {
      const int nn = e >> 7, k = e & 127;
      atomicAdd(&gacc[M_W4 + e], da4[nn] * bf2f(h3[k]));
    }
    for (int k = lane; k < 64; k += 32) atomicAdd(&gacc[M_B4 + k], da4[k]);
    for (int k = lane; k < 128; k += 32) {
      float s = 0.f;
      for (int nn = 0; nn < 64; ++nn) s += wgt(P.w + OFF_W4, K4, nn, k) * da4[nn];
      da3[k] = bf2f(h3[k]) > 0.f ? s : 0.f;
    }
    __syncwarp();
    // conv3 (h2 [32][4][4] bordered 6x6 -> da3 [32][2][2])
    for (int e = lane; e < 32 * 288; e += 32) {
      const int o2 = e / 288, k = e % 288, c = k / 9, u = (k % 9) / 3, v = k % 3;
      float s = 0.f;
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
          s += da3[o2 * 4 + i * 2 + j] * bf2f(h2[c * 36 + (2 * i + u) * 6 + (2 * j + v)]);
      atomicAdd(&gacc[M_W3 + e], s);
    }
    if (lane < 32)
      atomicAdd(&gacc[M_B3 + lane],
                da3[lane * 4] + da3[lane * 4 + 1] + da3[lane * 4 + 2] + da3[lane * 4 + 3]);
    // dh2[c][yy][xx] = sum over o, taps hitting (yy, xx)
    for (int e = lane; e < 32 * 16; e += 32) {
      const int c = e >> 4, yy = (e >> 2) & 3, xx = e & 3;
      float s = 0.f;
      for (int u = 0; u < 3; ++u) {
        const int ti = yy + 1 - u;
        if (ti < 0 || (ti & 1) || ti / 2 >= 2) continue;
        for (int v = 0; v < 3; ++v) {
          const int tj = xx + 1 - v;
          if (tj < 0 || (tj & 1) || tj / 2 >= 2) continue;
          const int i = ti / 2, j = tj / 2;
          for (int o2 = 0; o2 < 32; ++o2)
            s += wgt(P.w + OFF_W3, K3, o2, c * 9 + u * 3 + v) * da3[o2 * 4 + i * 2 + j];
        }
      }
      da2[e] = bf2f(h2[c * 36 + (yy + 1) * 6 + (xx + 1)]) > 0.f ? s : 0.f;
    }
    __syncwarp();
    // conv2 (h1 [32][8][8] bordered 10x10 -> da2 [32][4][4])
    for (int e = lane; e < 32 * 288; e += 32) {
      const int o2 = e / 288, k = e % 288, c = k / 9, u = (k % 9) / 3, v = k % 3;
      float s = 0.f;
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          s += da2[o2 * 16 + i * 4 + j] * bf2f(h1[c * 100 + (2 * i + u) * 10 + (2 * j + v)]);
      atomicAdd(&gacc[M_W2 + e], s);
    }
    {
      float s = 0.f;
      for (int q = 0; q < 16; ++q) s += da2[lane * 16 + q];
      atomicAdd(&gacc[M_B2 + lane], s);
    }
    for (int e = lane; e < 32 * 64; e += 32) {
      const int c = e >> 6, yy = (e >> 3) & 7, xx = e & 7;
      float s = 0.f;
      for (int u = 0; u < 3; ++u) {
        const int ti = yy + 1 - u;
        if (ti < 0 || (ti & 1) || ti / 2 >= 4) continue;
        for (int v = 0; v < 3; ++v) {
          const int tj = xx + 1 - v;
          if (tj < 0 || (tj & 1) || tj / 2 >= 4) continue;
          const int i = ti / 2, j = tj / 2;
          for (int o2 = 0; o2 < 32; ++o2)
            s += wgt(P.w + OFF_W2, K2, o2, c * 9 + u * 3 + v) * da2[o2 * 16 + i * 4 + j];
        }
      }
      da1[e] = bf2f(h1[c * 100 + (yy + 1) * 10 + (xx + 1)]) > 0.f ? s : 0.f;
    }
    __syncwarp();
    // conv1 (x [4][16][16] bordered 18x18 -> da1 [32][8][8])
    for (int e = lane; e < 32 * 36; e += 32) {
      const int o2 = e / 36, k = e % 36, c = k / 9, u = (k % 9) / 3, v = k % 3;
      float s = 0.f;
      for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j)
          s += da1[o2 * 64 + i * 8 + j] * bf2f(xb[c * 324 + (2 * i + u) * 18 + (2 * j + v)]);
      atomicAdd(&gacc[M_W1 + e], s);
    }
    {
      float s = 0.f;
      for (int q = 0; q < 64; ++q) s += da1[lane * 64 + q];
      atomicAdd(&gacc[M_B1 + lane], s);
    }
    __syncwarp();
  }
  if (lane == 0) atomicAdd(loss_sum, lsum);
  __syncthreads();
  for (int i = threadIdx.x; i < N_MASTER; i += blockDim.x)
    if (gacc[i] != 0.f) atomicAdd(&grad[i], gacc[i]);
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

int32_t* net_fault_word() {
  static int32_t* addr[64] = {};
  static PerDeviceOnce once;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  once_per_device(once, [&] {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_net_fault);
    addr[dev] = static_cast<int32_t*>(p);
    return e;
  });
  return addr[dev];
}

int initnet_train_smem() {
  return ((N_MASTER * 4 + 127) & ~127) + TRAIN_WARPS * WARP_SMEM + TRAIN_WARPS * BW_FLOATS * 4;
}

}  // namespace vio

extern "C" vio_status vio_initnet_pack(const float* d_master, void* d_packed, void* stream) {
  using namespace vio::net;
  if (!d_master || !d_packed) return VIO_ERR_INVALID_ARG;
  uint8_t* p = reinterpret_cast<uint8_t*>(d_packed);
  vio::pack_kernel<<<(N_BF16 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      d_master, reinterpret_cast<uint16_t*>(p), reinterpret_cast<float*>(p + OFF_B));
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" vio_status vio_initnet_extract(const vio_pyr_layout* layout, const vio_pyr_batch* src,
                                          const vio_pyr_batch* dst, const float* d_pts,
                                          const int32_t* d_count, int32_t capacity,
                                          int32_t level_a, int32_t level_b, uint16_t* d_x,
                                          void* stream) {
  if (!layout || !src || !dst || !d_pts || !d_x || capacity < 0 ||
      src->n_images != dst->n_images || src->n_images < 1)
    return VIO_ERR_INVALID_ARG;
  if (level_a < 0 || level_b < 0 || level_a >= layout->n_levels || level_b >= layout->n_levels)
    return VIO_ERR_INVALID_ARG;
  if ((layout->n_levels > 1) && (!src->d_upper || !dst->d_upper)) return VIO_ERR_INVALID_ARG;
  vio::ExtractArgs a{vio::make_geom(*layout), vio::make_batch(*src), vio::make_batch(*dst),
                     d_pts, d_count, capacity, level_a, level_b, d_x};
  const long long warps = (long long)capacity * src->n_images;
  if (warps == 0) return VIO_OK;
  vio::extract_kernel<<<(unsigned)((warps + 3) / 4), 128, 0, (cudaStream_t)stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" vio_status vio_initnet_forward(const void* d_packed, const uint16_t* d_x, int32_t n,
                                          float* d_out, void* stream) {
  using namespace vio::net;
  if (!d_packed || !d_x || !d_out || n < 0 || ((uintptr_t)d_packed & 15) ||
      ((uintptr_t)d_x & 15))
    return VIO_ERR_INVALID_ARG;
  if (n == 0) return VIO_OK;
  static vio::PerDeviceOnce attr;
  if (vio::once_per_device(attr, [] {
        return cudaFuncSetAttribute(vio::forward_tc_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, vio::ntc::SMEM);
      }) != cudaSuccess)
    return VIO_ERR_CUDA;
  const int rounds = (n + vio::ntc::ROUND - 1) / vio::ntc::ROUND, sms = vio::sm_count();
  vio::forward_tc_kernel<<<rounds < sms ? rounds : sms, vio::ntc::THREADS, vio::ntc::SMEM,
                           (cudaStream_t)stream>>>(d_packed, d_x, n, d_out,
                                                   vio::net_fault_word());
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" vio_status vio_initnet_fault(int32_t* status) {
  if (!status) return VIO_ERR_INVALID_ARG;
  int32_t* w = vio::net_fault_word();
  if (!w) return VIO_ERR_CUDA;
  int32_t v = 0;
  if (cudaMemcpy(&v, w, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(w, 0, sizeof(v)) != cudaSuccess)
    return VIO_ERR_CUDA;
  *status = v;
  return VIO_OK;
}

extern "C" vio_status vio_initnet_train_step(const void* d_packed, const uint16_t* d_x,
                                             const float* d_flow, const int32_t* d_index,
                                             int32_t n, float grad_scale, float label_radius,
                                             float* d_grad, float* d_loss, void* stream) {
  if (!d_packed || !d_x || !d_flow || !d_grad || !d_loss || n < 0 || !(label_radius > 0.f))
    return VIO_ERR_INVALID_ARG;
  if (n == 0) return VIO_OK;
  const int smem = vio::initnet_train_smem();
  cudaError_t e = cudaFuncSetAttribute(vio::train_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return VIO_ERR_CUDA;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)std::min<long long>((long long)sms, (n + vio::TRAIN_WARPS - 1) /
                                                                  vio::TRAIN_WARPS);
  vio::train_kernel<<<blocks, vio::TRAIN_WARPS * 32, smem, (cudaStream_t)stream>>>(
      d_packed, d_x, d_flow, d_index, n, grad_scale, label_radius, d_grad, d_loss);
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

extern "C" vio_status vio_initnet_adam(float* d_master, const float* d_grad, float* d_m,
                                       float* d_v, int32_t step, float lr, float beta1,
                                       float beta2, float eps, void* stream) {
  if (!d_master || !d_grad || !d_m || !d_v || step < 1) return VIO_ERR_INVALID_ARG;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  const int n = vio::net::N_MASTER;
  vio::adam_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
      d_master, d_grad, d_m, d_v, n, lr, beta1, beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}

static_assert(VIO_INITNET_N_PARAMS == vio::net::N_MASTER, "master parameter count");
static_assert(VIO_INITNET_PACKED_BYTES == vio::net::PACKED_BYTES, "packed size");
