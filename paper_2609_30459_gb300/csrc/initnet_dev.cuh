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

// ---------------------------------------------------------------------------
// Tiled inference: one CTA evaluates TT samples at a time, layer by layer,
// with the weights staged once per CTA in shared memory and every MMA tile
// filled with 16 rows (conv1: 64 positions x TT samples, conv2: 16 x TT,
// conv3: 4 x TT, dense layers: TT samples).
//
// Activations are channel-last (HWC) BF16 maps with a zero border, and the
// convolution weights are staged with their K axis in (tap, channel) order,
// so the two K values of an A-fragment register are two adjacent channels of
// one tap: one 32-bit shared load at an offset that is a compile-time
// constant of the K step plus the row's base. Pixel, row and sample strides
// are padded so that the 8 rows x 4 channel pairs of a fragment load hit 32
// distinct banks; weight rows are padded by 8 elements for the same reason.
// ---------------------------------------------------------------------------
constexpr int TT = 16;
constexpr int TILE_THREADS = 512;
constexpr int TILE_WARPS = TILE_THREADS / 32;
constexpr int PK1 = K1 + 8, PK2 = K2 + 8, PK3 = K3 + 8, PK4 = K4 + 8, PK5 = K5 + 8;
constexpr int SW1 = 0;
constexpr int SW2 = SW1 + N1 * PK1;
constexpr int SW3 = SW2 + N2 * PK2;
constexpr int SW4 = SW3 + N3 * PK3;
constexpr int SW5 = SW4 + N4 * PK4;
constexpr int SW_END = SW5 + N5 * PK5;          // elements
// map geometry (elements): pixel stride, row stride, sample stride
constexpr int X_PIX = 4, X_ROW = XP * X_PIX;                 // input 18 x 18 x 4
constexpr int H1_PIX = 36, H1_ROW = H1P * H1_PIX + 8;        // 10 x 10 x 32 (+pad)
constexpr int H1_SAMPLE = H1P * H1_ROW;
constexpr int H2_PIX = 36, H2_ROW = H2P * H2_PIX + 16;       // 6 x 6 x 32 (+pad)
constexpr int XR_SAMPLE = 1440;                              // input / H2 region per sample
constexpr int H3_SAMPLE = 136, H4_SAMPLE = 72;
static_assert(XP * X_ROW <= XR_SAMPLE && H2P * H2_ROW <= XR_SAMPLE, "region");
constexpr int T_W = 0;                                       // byte offsets
constexpr int T_B = T_W + SW_END * 2;
constexpr int T_X = ((T_B + N_BIAS * 4) + 15) & ~15;
constexpr int T_H1 = T_X + TT * XR_SAMPLE * 2;
constexpr int T_H3 = T_H1 + TT * H1_SAMPLE * 2;
constexpr int T_H4 = T_H3 + TT * H3_SAMPLE * 2;
constexpr int T_OUT = T_H4 + TT * H4_SAMPLE * 2;             // TT x 3 floats
constexpr int T_ZERO = T_OUT + TT * 3 * 4;
constexpr int TILE_SMEM = T_ZERO + 16;
static_assert(TILE_SMEM <= 227 * 1024, "tile shared memory");
// ldmatrix rows: 16-byte aligned weight rows and layer bases
static_assert((PK1 * 2) % 16 == 0 && (PK2 * 2) % 16 == 0 && (PK4 * 2) % 16 == 0 &&
                  (PK5 * 2) % 16 == 0 && (SW2 * 2) % 16 == 0 && (SW3 * 2) % 16 == 0 &&
                  (SW4 * 2) % 16 == 0 && (SW5 * 2) % 16 == 0 && T_W % 16 == 0,
              "ldmatrix alignment");

struct TileSmem {
  uint16_t* w;
  float* b;
  uint16_t* x;      // input, then conv2's output
  uint16_t* h1;
  uint16_t* h3;
  uint16_t* h4;
  float* out;
  const uint16_t* zero;
};

__device__ __forceinline__ TileSmem tile_smem(uint8_t* sm) {
  return TileSmem{reinterpret_cast<uint16_t*>(sm + T_W), reinterpret_cast<float*>(sm + T_B),
                  reinterpret_cast<uint16_t*>(sm + T_X), reinterpret_cast<uint16_t*>(sm + T_H1),
                  reinterpret_cast<uint16_t*>(sm + T_H3), reinterpret_cast<uint16_t*>(sm + T_H4),
                  reinterpret_cast<float*>(sm + T_OUT),
                  reinterpret_cast<const uint16_t*>(sm + T_ZERO)};
}

// Weights into padded rows (convolutions re-ordered to K = tap * CIN + c),
// biases, and zeros everywhere else (H1's border is never written again).
// Ends with a barrier.
__device__ __forceinline__ void tile_setup(const Packed& P, uint8_t* sm) {
  uint32_t* z = reinterpret_cast<uint32_t*>(sm + T_X);
  for (int i = threadIdx.x; i < (TILE_SMEM - T_X) / 4; i += blockDim.x) z[i] = 0u;
  uint32_t* zw = reinterpret_cast<uint32_t*>(sm + T_W + SW1 * 2);
  for (int i = threadIdx.x; i < N1 * PK1 / 2; i += blockDim.x) zw[i] = 0u;
  __syncthreads();
  const TileSmem S = tile_smem(sm);
  // convolutions: packed (n, c*9 + tap) -> staged (n, tap*CIN + c); reads
  // are coalesced words of the packed rows, the permutation is in the stores
  // (the padding columns 36..47 of conv1 stay zero from the clear above)
  for (int i = threadIdx.x; i < N1 * K1 / 2; i += blockDim.x) {
    const uint32_t v = __ldg(reinterpret_cast<const uint32_t*>(P.w + OFF_W1) + i);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = 2 * i + h, n = e / K1, kc = e - n * K1;
      const int c = kc / 9, tap = kc - 9 * c;
      if (kc < 36) S.w[SW1 + n * PK1 + tap * 4 + c] = (uint16_t)(v >> (16 * h));
    }
  }
  for (int i = threadIdx.x; i < N2 * K2; i += blockDim.x) {   // conv2 and conv3 words
    const int l = i >= N2 * K2 / 2, j = i - l * (N2 * K2 / 2);
    const uint32_t v = __ldg(reinterpret_cast<const uint32_t*>(P.w + (l ? OFF_W3 : OFF_W2)) + j);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = 2 * j + h, n = e / K2, kc = e - n * K2;
      const int c = kc / 9, tap = kc - 9 * c;
      S.w[(l ? SW3 : SW2) + n * PK2 + tap * 32 + c] = (uint16_t)(v >> (16 * h));
    }
  }
  // dense layers: rows as packed
  for (int i = threadIdx.x; i < N4 * K4 / 2; i += blockDim.x) {
    const int n = i / (K4 / 2), c = i - n * (K4 / 2);
    reinterpret_cast<uint32_t*>(S.w + SW4 + n * PK4)[c] =
        __ldg(reinterpret_cast<const uint32_t*>(P.w + OFF_W4) + i);
  }
  for (int i = threadIdx.x; i < N5 * K5 / 2; i += blockDim.x) {
    const int n = i / (K5 / 2), c = i - n * (K5 / 2);
    reinterpret_cast<uint32_t*>(S.w + SW5 + n * PK5)[c] =
        __ldg(reinterpret_cast<const uint32_t*>(P.w + OFF_W5) + i);
  }
  for (int i = threadIdx.x; i < N_BIAS; i += blockDim.x) S.b[i] = __ldg(P.b + i);
  __syncthreads();
}

__device__ __forceinline__ uint32_t lds32(const uint16_t* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// B fragments of two n-tiles (rows n0 .. n0+15 of a weight matrix W[n][k]
// with row stride PK, columns k0 .. k0+15) by one ldmatrix: b[0], b[1] for
// n-tile n0, b[2], b[3] for n0 + 8. Rows are 16-byte aligned (PK * 2 and k0
// * 2 multiples of 16).
__device__ __forceinline__ void ldsm_b2(uint32_t (&b)[4], const uint16_t* W, int PK, int n0,
                                        int k0, int lane) {
  const int m = lane >> 3, row = lane & 7;
  const uint16_t* p = W + (n0 + (m >> 1) * 8 + row) * PK + k0 + (m & 1) * 8;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3])
               : "r"(a));
}

// B fragment of one n-tile (rows n0 .. n0+7, columns k0 .. k0+15).
__device__ __forceinline__ void ldsm_b1(uint32_t (&b)[2], const uint16_t* W, int PK, int n0,
                                        int k0, int lane) {
  const int m = (lane >> 3) & 1, row = lane & 7;
  const uint16_t* p = W + (n0 + row) * PK + k0 + m * 8;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(b[0]), "=r"(b[1])
               : "r"(a));
}

// Epilogue of one accumulator tile: bias, ReLU, BF16 pairs (n, n+1) stored as
// one word at out_row[h] + n (the caller's per-row base).
__device__ __forceinline__ void store_pairs(const float (&acc)[4], const float* bias, int n0,
                                            uint16_t* row0, uint16_t* row1) {
  const float b0 = bias[n0], b1 = bias[n0 + 1];
  const uint32_t lo = (uint32_t)f2bf(fmaxf(acc[0] + b0, 0.f)) |
                      ((uint32_t)f2bf(fmaxf(acc[1] + b1, 0.f)) << 16);
  const uint32_t hi = (uint32_t)f2bf(fmaxf(acc[2] + b0, 0.f)) |
                      ((uint32_t)f2bf(fmaxf(acc[3] + b1, 0.f)) << 16);
  *reinterpret_cast<uint32_t*>(row0 + n0) = lo;
  *reinterpret_cast<uint32_t*>(row1 + n0) = hi;
}

// conv1 on one M tile: rows mt*16.. of TT*64 (sample, 8x8 position), all 32
// output channels into H1 (HWC).
__device__ __forceinline__ void tile_conv1(const TileSmem& S, int mt, int lane) {
  const int g = lane >> 2, t = lane & 3;
  int base[2];
  uint16_t* orow[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = mt * 16 + g + 8 * h, s = r >> 6, p = r & 63, i = p >> 3, j = p & 7;
    base[h] = s * XR_SAMPLE + (2 * i) * X_ROW + (2 * j) * X_PIX;
    orow[h] = S.h1 + s * H1_SAMPLE + (i + 1) * H1_ROW + (j + 1) * H1_PIX;
  }
  float acc[4][4] = {};
#pragma unroll
  for (int ks = 0; ks < K1 / 16; ++ks) {
    // lane's K pairs: taps 4 ks + t/2 and that + 2, channels 2 (t & 1) + {0, 1}
    uint32_t a[4];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int tap = 4 * ks + (t >> 1) + 2 * half;
      const int off = (tap / 3) * X_ROW + (tap % 3) * X_PIX + 2 * (t & 1);
#pragma unroll
      for (int h = 0; h < 2; ++h)
        a[h + 2 * half] = tap < 9 ? lds32(S.x + base[h] + off) : 0u;
    }
#pragma unroll
    for (int q = 0; q < 4; q += 2) {
      uint32_t b[4];
      ldsm_b2(b, S.w + SW1, PK1, q * 8, ks * 16, lane);
      mma16816(acc[q], a, b[0], b[1]);
      mma16816(acc[q + 1], a, b[2], b[3]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) store_pairs(acc[q], S.b + OFF_B1, q * 8 + 2 * t, orow[0], orow[1]);
}

// conv2 on one sample's 16 positions (one M tile), all 32 channels into the
// X region as H2 (HWC, 6x6 bordered).
__device__ __forceinline__ void tile_conv2(const TileSmem& S, int s, int lane) {
  const int g = lane >> 2, t = lane & 3;
  int base[2];
  uint16_t* orow[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int p = g + 8 * h, i = p >> 2, j = p & 3;
    base[h] = s * H1_SAMPLE + (2 * i) * H1_ROW + (2 * j) * H1_PIX + 2 * t;
    orow[h] = S.x + s * XR_SAMPLE + (i + 1) * H2_ROW + (j + 1) * H2_PIX;
  }
  float acc[4][4] = {};
#pragma unroll
  for (int ks = 0; ks < K2 / 16; ++ks) {
    const int tap = ks >> 1, c0 = (ks & 1) * 16;
    const int off = (tap / 3) * H1_ROW + (tap % 3) * H1_PIX + c0;
    uint32_t a[4];
    a[0] = lds32(S.h1 + base[0] + off);
    a[1] = lds32(S.h1 + base[1] + off);
    a[2] = lds32(S.h1 + base[0] + off + 8);
    a[3] = lds32(S.h1 + base[1] + off + 8);
#pragma unroll
    for (int q = 0; q < 4; q += 2) {
      uint32_t b[4];
      ldsm_b2(b, S.w + SW2, PK2, q * 8, ks * 16, lane);
      mma16816(acc[q], a, b[0], b[1]);
      mma16816(acc[q + 1], a, b[2], b[3]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) store_pairs(acc[q], S.b + OFF_B2, q * 8 + 2 * t, orow[0], orow[1]);
}

// conv3 on one M tile (4 samples x 2x2 positions), one n-tile, into H3 as
// (channel, row, column) vectors.
__device__ __forceinline__ void tile_conv3(const TileSmem& S, int mt, int nt, int lane) {
  const int g = lane >> 2, t = lane & 3;
  int base[2], orow[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = mt * 16 + g + 8 * h, s = r >> 2, p = r & 3, i = p >> 1, j = p & 1;
    base[h] = s * XR_SAMPLE + (2 * i) * H2_ROW + (2 * j) * H2_PIX + 2 * t;
    orow[h] = s * H3_SAMPLE + p;
  }
  // two accumulators (the two channel halves of each tap): two independent
  // MMA chains of nine instead of one of eighteen
  float acc[2][4] = {};
#pragma unroll
  for (int ks = 0; ks < K3 / 16; ++ks) {
    const int tap = ks >> 1, c0 = (ks & 1) * 16;
    const int off = (tap / 3) * H2_ROW + (tap % 3) * H2_PIX + c0;
    uint32_t a[4];
    a[0] = lds32(S.x + base[0] + off);
    a[1] = lds32(S.x + base[1] + off);
    a[2] = lds32(S.x + base[0] + off + 8);
    a[3] = lds32(S.x + base[1] + off + 8);
    uint32_t b[2];
    ldsm_b1(b, S.w + SW3, PK3, nt * 8, ks * 16, lane);
    mma16816(acc[ks & 1], a, b[0], b[1]);
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int n = nt * 8 + 2 * t + (e & 1);
    S.h3[orow[e >> 1] + n * 4] = f2bf(fmaxf(acc[0][e] + acc[1][e] + S.b[OFF_B3 + n], 0.f));
  }
}

// Dense layer over the TT samples (rows), n-tile nt.
template <int K, int PK, int STRIDE>
__device__ __forceinline__ void fc_ntile(const uint16_t* in, const uint16_t* W, int nt, int lane,
                                         float (&acc)[4]) {
  const int g = lane >> 2, t = lane & 3;
  float part[2][4] = {};        // even and odd K steps: two independent chains
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    uint32_t a[4];
    a[0] = lds32(in + g * STRIDE + ks * 16 + 2 * t);
    a[1] = lds32(in + (g + 8) * STRIDE + ks * 16 + 2 * t);
    a[2] = lds32(in + g * STRIDE + ks * 16 + 2 * t + 8);
    a[3] = lds32(in + (g + 8) * STRIDE + ks * 16 + 2 * t + 8);
    uint32_t b[2];
    ldsm_b1(b, W, PK, nt * 8, ks * 16, lane);
    mma16816(part[ks & 1], a, b[0], b[1]);
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) acc[e] = part[0][e] + part[1][e];
}

// Zero border pixels of the input maps (the region held conv2's output).
__device__ __forceinline__ void tile_clear_input_border(const TileSmem& S) {
  for (int i = threadIdx.x; i < TT * 68; i += blockDim.x) {
    const int s = i / 68, k = i - s * 68;
    const int y = k < 18 ? 0 : (k < 36 ? 17 : 1 + (k - 36) / 2);
    const int x = k < 36 ? k % 18 : ((k - 36) & 1) * 17;
    *reinterpret_cast<uint2*>(S.x + s * XR_SAMPLE + y * X_ROW + x * X_PIX) = make_uint2(0u, 0u);
  }
}

// conv1, conv2 and conv3 of the TT inputs in S.x (interior written by the
// caller and the border cleared by tile_clear_input_border, then a barrier):
// H3 in S.h3. Ends with a barrier, after which S.x is free.
__device__ __forceinline__ void tile_convs(const TileSmem& S) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int mt = warp; mt < TT * 4; mt += TILE_WARPS) tile_conv1(S, mt, lane);
  __syncthreads();
  // conv2 writes into the input region: clear its border pixels first
  // (20 per sample, 32 channels = 8 words each)
  for (int i = threadIdx.x; i < TT * 20 * 8; i += blockDim.x) {
    const int s = i / 160, r = i - s * 160, k = r >> 3, w4 = r & 7;
    const int y = k < 6 ? 0 : (k < 12 ? 5 : 1 + (k - 12) / 2);
    const int x = k < 12 ? k % 6 : ((k - 12) & 1) * 5;
    *reinterpret_cast<uint2*>(S.x + s * XR_SAMPLE + y * H2_ROW + x * H2_PIX + 4 * w4) =
        make_uint2(0u, 0u);
  }
  for (int s = warp; s < TT; s += TILE_WARPS) tile_conv2(S, s, lane);
  __syncthreads();
  for (int it = warp; it < (TT / 4) * 4; it += TILE_WARPS) tile_conv3(S, it >> 2, it & 3, lane);
  __syncthreads();
}

// fc1, one n-tile of 8 outputs per warp (warps 0..7): H3 -> H4. The caller
// places the barrier before fc2.
__device__ __forceinline__ void tile_fc1(const TileSmem& S, int warp, int lane) {
  const int g = lane >> 2, t = lane & 3;
  float acc[4];
  fc_ntile<K4, PK4, H3_SAMPLE>(S.h3, S.w + SW4, warp, lane, acc);
  store_pairs(acc, S.b + OFF_B4, warp * 8 + 2 * t, S.h4 + g * H4_SAMPLE,
              S.h4 + (g + 8) * H4_SAMPLE);
}

// fc2 by one warp: out(sample, n, value) for the TT samples and n < 3, value
// (dx, dy, conf) = (16 o0, 16 o1, sigmoid(o2)).
template <class Out>
__device__ __forceinline__ void tile_fc2(const TileSmem& S, int lane, Out out) {
  const int g = lane >> 2, t = lane & 3;
  float acc[4];
  fc_ntile<K5, PK5, H4_SAMPLE>(S.h4, S.w + SW5, 0, lane, acc);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int row = g + 8 * (e >> 1), n = 2 * t + (e & 1);
    if (n < 3) {
      const float o = acc[e] + S.b[OFF_B5 + n];
      out(row, n, n < 2 ? o * kScale : 1.f / (1.f + expf(-o)));
    }
  }
}

// The network on the TT inputs in S.x (as for tile_convs); results
// (dx, dy, conf) in S.out[3 s ..]. Ends with a barrier.
__device__ __forceinline__ void tile_forward(const TileSmem& S) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  tile_convs(S);
  if (warp < 8) tile_fc1(S, warp, lane);
  __syncthreads();
  if (warp == 0) tile_fc2(S, lane, [&](int row, int n, float v) { S.out[row * 3 + n] = v; });
  __syncthreads();
}

// Writes row r (0..15) of channel ch of sample s's input map from the level
// images: 16 values (v - 128) / 64 of the integer grid of keypoint (px, py),
// 0 outside the level (the sampling of extract_warp).
__device__ __forceinline__ void tile_input_row(const TileSmem& S, int s, int ch, int r,
                                               const Geom& g, const Batch& src, int src_img,
                                               const Batch& dst, int dst_img, float px,
                                               float py, int la, int lb) {
  const int lv = ch < 2 ? la : lb;
  const float sc = __int_as_float((127 - lv) << 23);
  const int cx = (int)floorf(px * sc + 0.5f) - 8;
  const int cy = (int)floorf(py * sc + 0.5f) - 8 + r;
  const bool in_row = cy >= 0 && cy < g.h[lv];
  const uint8_t* row = nullptr;
  if (in_row)
    row = level_ptr(g, (ch & 1) ? dst : src, (ch & 1) ? dst_img : src_img, lv) +
          (long long)cy * g.pitch[lv];
  uint8_t v[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const int x = cx + c;
    v[c] = (in_row && x >= 0 && x < g.w[lv]) ? __ldg(row + x) : (uint8_t)128;
  }
  uint16_t* out = S.x + s * XR_SAMPLE + (r + 1) * X_ROW + X_PIX + ch;
#pragma unroll
  for (int c = 0; c < 16; ++c) out[c * X_PIX] = f2bf(((float)v[c] - 128.f) * (1.f / 64.f));
}


// Prefetch of one input row into registers, so that the loads of the next
// tile are in flight while the current tile computes: the five aligned
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

__device__ __forceinline__ void row_store(const RowWords& R, const TileSmem& S, int s, int ch,
                                          int r) {
  uint16_t* out = S.x + s * XR_SAMPLE + (r + 1) * X_ROW + X_PIX + ch;
  const unsigned sh = 8u * (unsigned)(R.cx - R.x4);
  uint32_t a[4];      // the 16 pixels, aligned to the row's first pixel
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = __funnelshift_r(R.w[k], R.w[k + 1], sh);
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    const int x = R.cx + c;
    uint32_t v = (a[c >> 2] >> (8 * (c & 3))) & 0xffu;
    if (!R.row_ok || x < 0 || x >= R.wl) v = 128u;
    out[c * X_PIX] = f2bf(((float)v - 128.f) * (1.f / 64.f));
  }
}

}  // namespace net
}  // namespace vio
