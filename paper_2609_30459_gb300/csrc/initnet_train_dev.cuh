// Device code of the flow network's training pass (the train kernel of
// initnet.cu): per warp, one sample at a time, the forward pass with BF16
// activations (forward_warp), the loss of the flow and confidence outputs,
// and the backward pass in FP32, the weight gradients summed in shared
// memory per CTA and added to the global gradient once per CTA.
#pragma once
#include <math.h>

#include "initnet_dev.cuh"

namespace vio {
namespace net {

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

constexpr int TRAIN_WARPS = 4;
// per-warp FP32 backward scratch: da4[64], da3[128], da2[512], da1[2048]
constexpr int BW_FLOATS = 64 + 128 + 512 + 2048;

__device__ __forceinline__ float wgt(const uint16_t* W, int K, int n, int k) {
  return bf2f(W[n * K + k]);
}

// Shared memory of one training CTA: the gradient accumulator, each warp's
// activations and its FP32 backward scratch.
constexpr int train_smem_bytes() {
  return ((N_MASTER * 4 + 127) & ~127) + TRAIN_WARPS * WARP_SMEM + TRAIN_WARPS * BW_FLOATS * 4;
}

// The training pass of one CTA of TRAIN_WARPS warps over samples blockIdx.x *
// TRAIN_WARPS + warp, stepping by gridDim.x * TRAIN_WARPS; dsm: the CTA's
// shared memory (train_smem_bytes()).
__device__ __forceinline__ void train_block(const void* __restrict__ packed_w,
                                            const uint16_t* __restrict__ x,
                                            const float* __restrict__ flow,
                                            const int32_t* __restrict__ index, int n,
                                            float grad_scale, float radius,
                                            float* __restrict__ grad,
                                            float* __restrict__ loss_sum, uint8_t* dsm) {
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

}  // namespace net
}  // namespace vio
