// Device code of the learned flow initializer (not in the paper; its
// initialisation uses the camera model and a predicted pose, Sec. III-E).
//
// Network: input 4 x 16 x 16 (source and target patch at pyramid levels a and
// b, integer grid around the keypoint, (v - 128) / 64), three 3x3 stride-2
// convolutions with 32 channels and ReLU (16 -> 8 -> 4 -> 2), flatten to 128,
// fully connected 128 -> 64 with ReLU, then 64 -> 3: flow = 16 px * (o0, o1)
// and confidence = sigmoid(o2).
//
// One warp evaluates one sample on the tensor cores: every layer is a GEMM
// (output positions x input taps) x (input taps x output channels) done with
// mma.sync m16n8k16 on BF16 operands and FP32 accumulators. Activations live
// in the warp's shared memory as BF16 with a zero border, so the im2col
// offset of (position, tap) splits into a per-row base plus a per-column
// offset and needs no bounds test. Weights are packed as BF16 [N][K] rows
// (K padded to a multiple of 16) so a B fragment is one 32-bit load.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"

namespace vio {
namespace net {

constexpr float kScale = 16.f;
// packed BF16 weight matrices [N][K] (element offsets) and FP32 biases
constexpr int K1 = 48, K2 = 288, K3 = 288, K4 = 128, K5 = 64;
constexpr int N1 = 32, N2 = 32, N3 = 32, N4 = 64, N5 = 8;
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + N1 * K1;   // 1536
constexpr int OFF_W3 = OFF_W2 + N2 * K2;   // 10752
constexpr int OFF_W4 = OFF_W3 + N3 * K3;   // 19968
constexpr int OFF_W5 = OFF_W4 + N4 * K4;   // 28160
constexpr int N_BF16 = OFF_W5 + N5 * K5;   // 28672
constexpr int OFF_B = N_BF16 * 2;          // byte offset of the biases
constexpr int OFF_B1 = 0, OFF_B2 = 32, OFF_B3 = 64, OFF_B4 = 96, OFF_B5 = 160;
constexpr int N_BIAS = 168;
constexpr int PACKED_BYTES = OFF_B + N_BIAS * 4;
// FP32 master parameters in the order w1 (32,4,3,3), b1, w2 (32,32,3,3), b2,
// w3, b3, w4 (64,128), b4, w5 (3,64), b5
constexpr int M_W1 = 0, M_B1 = 1152, M_W2 = 1184, M_B2 = 10400, M_W3 = 10432, M_B3 = 19648,
              M_W4 = 19680, M_B4 = 27872, M_W5 = 27936, M_B5 = 28128, N_MASTER = 28131;

// Per-warp shared memory (bytes): activations with a zero border.
constexpr int XP = 18;                   // input 16 + 2
constexpr int H1P = 10;                  // 8 + 2
constexpr int H2P = 6;                   // 4 + 2
constexpr int S_X = 0;                   // [4][18][18] bf16
constexpr int S_H1 = S_X + 4 * XP * XP * 2;          // 2592: [32][10][10]
constexpr int S_H2 = S_H1 + 32 * H1P * H1P * 2;      // +6400: [32][6][6]
constexpr int S_H3 = S_H2 + 32 * H2P * H2P * 2;      // +2304: [128]
constexpr int S_H4 = S_H3 + 128 * 2;                 // [64]
constexpr int S_ZERO = S_H4 + 64 * 2;                // 16 zero bytes (padding taps)
constexpr int WARP_SMEM = ((S_ZERO + 16) + 127) & ~127;

struct Packed {
  const uint16_t* w;   // N_BF16 bf16 bits
  const float* b;      // N_BIAS floats
};

__device__ __forceinline__ Packed packed(const void* p) {
  return Packed{reinterpret_cast<const uint16_t*>(p),
                reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(p) + OFF_B)};
}

__device__ __forceinline__ uint16_t f2bf(float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float bf2f(uint16_t v) {
  return __bfloat162float(__ushort_as_bfloat16(v));
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Offset of tap k (k = c*9 + u*3 + v) in a bordered [C][P][P] map, or -1
// beyond the real taps (the padding columns of K).
__device__ __forceinline__ int tap_off(int k, int ntaps, int P) {
  if (k >= ntaps) return -1;
  const int c = k / 9, r = k - 9 * c;
  const int u = r / 3, v = r - 3 * u;
  return c * P * P + u * P + v;
}

// 3x3 stride-2 convolution + bias + ReLU of a bordered BF16 map
// [CIN][HIN+2][HIN+2] into a bordered map [32][HOUT+2][HOUT+2] (or, when
// flat_out, into a plain [32*HOUT*HOUT] vector in (channel, row, col) order).
template <int CIN, int HIN, int KPAD, bool FLAT_OUT>
__device__ __forceinline__ void conv_layer(const uint16_t* in, uint16_t* out, const uint16_t* zero,
                                           const uint16_t* W, const float* bias, int lane) {
  constexpr int HOUT = HIN / 2;
  constexpr int P = HIN + 2, PO = HOUT + 2;
  constexpr int M = HOUT * HOUT;
  constexpr int MT = (M + 15) / 16;
  constexpr int NTAPS = CIN * 9;
  const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
  for (int mt = 0; mt < MT; ++mt) {
    // the two output positions (rows) of this thread in the tile
    int base[2];
    bool live[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = mt * 16 + g + 8 * h;
      live[h] = r < M;
      const int i = live[h] ? r / HOUT : 0, j = live[h] ? r % HOUT : 0;
      base[h] = 2 * i * P + 2 * j;     // bordered coordinates of tap (0, 0)
    }
    float acc[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll 2
    for (int ks = 0; ks < KPAD / 16; ++ks) {
      int off[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) off[q] = tap_off(ks * 16 + 2 * t + (q & 1) + 8 * (q >> 1),
                                                   NTAPS, P);
      uint32_t a[4];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
          const int q0 = 2 * half, q1 = 2 * half + 1;
          const uint16_t lo = (live[h] && off[q0] >= 0) ? in[base[h] + off[q0]] : zero[0];
          const uint16_t hi = (live[h] && off[q1] >= 0) ? in[base[h] + off[q1]] : zero[0];
          a[h + 2 * half] = (uint32_t)lo | ((uint32_t)hi << 16);
        }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const uint16_t* wr = W + (nt * 8 + g) * KPAD + ks * 16 + 2 * t;
        const uint32_t b0 = __ldg(reinterpret_cast<const uint32_t*>(wr));
        const uint32_t b1 = __ldg(reinterpret_cast<const uint32_t*>(wr + 8));
        mma16816(acc[nt], a, b0, b1);
      }
    }
    // epilogue: bias, ReLU, BF16
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = mt * 16 + g + 8 * (e >> 1);
        const int n = nt * 8 + 2 * t + (e & 1);
        if (r < M) {
          const float v = fmaxf(acc[nt][e] + bias[n], 0.f);
          const int i = r / HOUT, j = r % HOUT;
          if (FLAT_OUT)
            out[n * M + r] = f2bf(v);
          else
            out[n * PO * PO + (i + 1) * PO + (j + 1)] = f2bf(v);
        }
      }
  }
}

// Fully connected layer on one input vector (row 0 of a 16-row tile):
// out[n] = act(sum_k W[n][k] in[k] + b[n]) for n < NOUT; returns outputs in
// FP32 through `res` (thread-local: lanes with g == 0 hold row 0).
template <int K, int NT>
__device__ __forceinline__ void fc_layer(const uint16_t* in, const uint16_t* W, int lane,
                                         float (&acc)[NT][4]) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    uint32_t a[4] = {0u, 0u, 0u, 0u};
    if (g == 0) {
      const uint32_t* p = reinterpret_cast<const uint32_t*>(in + ks * 16 + 2 * t);
      a[0] = p[0];
      a[2] = p[4];
    }
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      const uint16_t* wr = W + (nt * 8 + g) * K + ks * 16 + 2 * t;
      const uint32_t b0 = __ldg(reinterpret_cast<const uint32_t*>(wr));
      const uint32_t b1 = __ldg(reinterpret_cast<const uint32_t*>(wr + 8));
      mma16816(acc[nt], a, b0, b1);
    }
  }
}

// Zero the borders (and the zero word) of a warp's activation buffers.
__device__ __forceinline__ void clear_warp_smem(uint8_t* ws, int lane) {
  uint32_t* p = reinterpret_cast<uint32_t*>(ws);
  for (int i = lane; i < WARP_SMEM / 4; i += 32) p[i] = 0u;
  __syncwarp();
}

// Forward pass of one sample whose input is in ws + S_X (bordered, BF16).
// Returns o[0..2] (raw outputs) in every lane.
__device__ __forceinline__ void forward_warp(const Packed& P, uint8_t* ws, int lane, float* o) {
  uint16_t* x = reinterpret_cast<uint16_t*>(ws + S_X);
  uint16_t* h1 = reinterpret_cast<uint16_t*>(ws + S_H1);
  uint16_t* h2 = reinterpret_cast<uint16_t*>(ws + S_H2);
  uint16_t* h3 = reinterpret_cast<uint16_t*>(ws + S_H3);
  uint16_t* h4 = reinterpret_cast<uint16_t*>(ws + S_H4);
  const uint16_t* zero = reinterpret_cast<const uint16_t*>(ws + S_ZERO);
  conv_layer<4, 16, K1, false>(x, h1, zero, P.w + OFF_W1, P.b + OFF_B1, lane);
  __syncwarp();
  conv_layer<32, 8, K2, false>(h1, h2, zero, P.w + OFF_W2, P.b + OFF_B2, lane);
  __syncwarp();
  conv_layer<32, 4, K3, true>(h2, h3, zero, P.w + OFF_W3, P.b + OFF_B3, lane);
  __syncwarp();
  const int g = lane >> 2, t = lane & 3;
  {
    float acc[8][4];
    fc_layer<K4, 8>(h3, P.w + OFF_W4, lane, acc);
    if (g == 0)
#pragma unroll
      for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int n = nt * 8 + 2 * t + e;
          h4[n] = f2bf(fmaxf(acc[nt][e] + P.b[OFF_B4 + n], 0.f));
        }
  }
  __syncwarp();
  float acc5[1][4];
  fc_layer<K5, 1>(h4, P.w + OFF_W5, lane, acc5);
  // row 0, columns 2t, 2t+1 live in lane t (g == 0): outputs 0..2 in lanes 0, 1
  const float v0 = acc5[0][0], v1 = acc5[0][1];
  const float a0 = __shfl_sync(0xffffffffu, v0, 0), a1 = __shfl_sync(0xffffffffu, v1, 0);
  const float a2 = __shfl_sync(0xffffffffu, v0, 1);
  o[0] = a0 + P.b[OFF_B5 + 0];
  o[1] = a1 + P.b[OFF_B5 + 1];
  o[2] = a2 + P.b[OFF_B5 + 2];
}

// Input of keypoint (px, py): for level l in (la, lb), the 16 x 16 integer
// grid from round(p / 2^l) - 8, source then target, (v - 128) / 64, zero
// outside the level; written bordered into ws + S_X.
__device__ __forceinline__ void extract_warp(const Geom& g, const Batch& src, int src_img,
                                             const Batch& dst, int dst_img, float px, float py,
                                             int la, int lb, uint8_t* ws, int lane) {
  uint16_t* x = reinterpret_cast<uint16_t*>(ws + S_X);
  for (int e = lane; e < 4 * 256; e += 32) {
    const int ch = e >> 8, rc = e & 255, r = rc >> 4, c = rc & 15;
    const int lv = ch < 2 ? la : lb;
    const Batch& b = (ch & 1) ? dst : src;
    const int img = (ch & 1) ? dst_img : src_img;
    const float sc = __int_as_float((127 - lv) << 23);
    const int cx = (int)floorf(px * sc + 0.5f) - 8 + c;
    const int cy = (int)floorf(py * sc + 0.5f) - 8 + r;
    float v = 0.f;
    if (cx >= 0 && cx < g.w[lv] && cy >= 0 && cy < g.h[lv])
      v = ((float)__ldg(level_ptr(g, b, img, lv) + (long long)cy * g.pitch[lv] + cx) - 128.f) *
          (1.f / 64.f);
    x[ch * XP * XP + (r + 1) * XP + (c + 1)] = f2bf(v);
  }
  __syncwarp();
}

}  // namespace net
}  // namespace vio

namespace vio {
namespace net {

// Prefetch of one input row into registers, so that the loads of the next
// group are in flight while the current one computes: the five aligned
// 32-bit words that cover the row's 16 pixels. Only for upper pyramid levels
// (rows start 128-byte aligned and the pitch is a multiple of 128 bytes, so
// a word that starts inside the level lies inside the row's pitch).
struct RowWords {
  uint32_t w[5];
  int cx, x4, wl;     // first pixel, first word's pixel, level width
  bool row_ok;        // the row lies inside the level
};

__device__ __forceinline__ void row_prefetch(RowWords& R, const Geom& g, const Batch& b, int img,
                                             int lv, float px, float py, int r) {
  const float sc = __int_as_float((127 - lv) << 23);
  R.cx = (int)floorf(px * sc + 0.5f) - 8;
  const int cy = (int)floorf(py * sc + 0.5f) - 8 + r;
  R.wl = g.w[lv];
  R.row_ok = cy >= 0 && cy < g.h[lv];
  R.x4 = R.cx & ~3;
  const uint8_t* row = level_ptr(g, b, img, lv) + (long long)(R.row_ok ? cy : 0) * g.pitch[lv];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int x = R.x4 + 4 * k;
    R.w[k] = (R.row_ok && x >= 0 && x < R.wl)
                 ? __ldg(reinterpret_cast<const uint32_t*>(row + x)) : 0x80808080u;
  }
}

}  // namespace net
}  // namespace vio
