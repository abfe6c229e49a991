// Forward pass of the flow initializer on the fifth-generation tensor cores
// (tcgen05): every layer is a sum of M = 128-row MMAs with BF16 operands in
// shared memory and the FP32 accumulator in tensor memory; the epilogues
// (bias, ReLU, BF16) read the accumulator back and write the next layer's
// operand. Same network and arithmetic as initnet_dev.cuh (BF16 weights and
// activations, FP32 sums), in another summation order.
//
// A CTA of EPI_WARPS + 1 warps runs rounds of 32 samples (EPI_WARPS warps stage
// inputs and drain the accumulators; the last one issues the MMAs):
//
//   conv1  per group of 8 samples: 4 tiles of 16 positions (two output rows)
//          x 8 samples; a row's K = 3 tap rows x 16 (the 3 taps of a kernel
//          row and a zero-weighted fourth, x 4 channels)   -> 4 x 3 MMAs, N 32
//   conv2  per group: 16 positions x 8 samples, K = 9 taps x 32 channels
//                                                          -> 18 MMAs, N 32
//   conv3  per round: 4 positions x 32 samples, K = 9 x 32 -> 18 MMAs, N 32
//   fc1    per round: rows = the 32 samples (96 rows unused), K 128 -> 8, N 64
//   fc2    per round: K 64, N 16 (3 used)                  -> 4 MMAs
//
// Stride-2 3x3 convolutions need no im2col: a layer's input is stored in
// "phase maps", so that for every tap the 128 rows of the A operand sit at
// one fixed stride (16 bytes) from a tap-dependent start. For a bordered input
// map (border 1 = the zero padding) the output (i, j) reads pixel
// (2i + u, 2j + v) for tap (u, v); pixels split by row parity pu = Y % 2 and
// by column into three maps: even columns at X / 2 (tap v = 0), odd columns
// at X / 2 (v = 1) and even columns at X / 2 - 1 (v = 2). In each map the
// entry of output (i, j) for tap row u sits at map row i + u / 2 and column j,
// so (row, column, sample) order makes the A rows of a tap contiguous. With
// the sample as the fastest index, the 8 lanes of a 16-byte store phase (8
// samples) write 8 different bank groups in every epilogue and input store.
// conv1's input (4 channels, 8 bytes per pixel) pairs the pixels instead:
// one 16-byte entry holds pixels X and X + 1, in an even-start map (taps 0,
// 1) and a map shifted by two pixels (tap 2 and the unused X + 3).
#pragma once
#include "initnet_dev.cuh"
#include "tc05.cuh"

namespace vio {

// Device address of the forward passes' status word (per device; null if the
// lookup fails).
int32_t* net_fault_word();

namespace ntc {

constexpr int EPI_WARPS = 4;                       // epilogue / input warps (4 or 8)
constexpr int NH = EPI_WARPS / 4;                  // epilogue warps per accumulator lane quarter
constexpr int THREADS = 32 * (EPI_WARPS + 1);      // + one MMA-issuing warp
constexpr int ROUND = 32;     // samples per round
constexpr int GROUP = 8;      // samples per conv1/conv2 group

// Shared memory (byte offsets). B operands: [K chunk][N group][8 rows][16 B].
constexpr int W1_OFF = 0;                      // 3 tap rows x (N 32, K 16)
constexpr int W2_OFF = W1_OFF + 3 * 1024;      // 9 taps x 2 K halves x (N 32, K 16)
constexpr int W3_OFF = W2_OFF + 18 * 1024;
constexpr int W4_OFF = W3_OFF + 18 * 1024;     // N 64, K 128 (K in position-major order)
constexpr int W5_OFF = W4_OFF + 16 * 1024;     // N 16, K 64
// conv1 input: [pu 2][shift 2][row 9][col 8][sample 8][16 B]
constexpr int P_OFF = W5_OFF + 2 * 1024;
constexpr int P_MAP = 9 * 8 * 8 * 16, P_ROW = 8 * 8 * 16;
// conv1 output = conv2 input: [map 6][K chunk 4][row 5][col 4][sample 8][16 B]
constexpr int H1_OFF = P_OFF + 4 * P_MAP;
constexpr int H1_CHUNK = 5 * 4 * 8 * 16, H1_MAP = 4 * H1_CHUNK;
// conv2 output = conv3 input: [map 6][K chunk 4][row 3][col 2][sample 32][16 B]
constexpr int H2_OFF = H1_OFF + 6 * H1_MAP;
constexpr int H2_CHUNK = 3 * 2 * 32 * 16, H2_MAP = 4 * H2_CHUNK;
// conv3 output and fc1 output (the A operands of fc1 and fc2) share conv1's
// input region (free once a round's conv layers are done): [K chunk][row
// group 4][8 rows][16 B], the 96 unused rows of the M = 128 MMA read the next
// chunks (and 1.5 KB after the last one)
constexpr int H3_OFF = P_OFF;
constexpr int H4_OFF = P_OFF + 16 * 512 + 1536;
constexpr int BIAS_OFF = H2_OFF + 6 * H2_MAP;
constexpr int BAR_OFF = BIAS_OFF + net::N_BIAS * 4;
constexpr int N_BARS = 10;
constexpr int SLOT_OFF = BAR_OFF + 8 * N_BARS;    // tensor-memory address, abort flag
constexpr int SMEM = SLOT_OFF + 8;
static_assert(H4_OFF + 8 * 512 + 1536 <= P_OFF + 4 * P_MAP, "fc operands inside conv1's input");
static_assert(BAR_OFF % 8 == 0, "mbarrier alignment");

// Tensor-memory columns of the accumulators (conv1 and conv2 double-buffered
// by group parity).
constexpr int C1 = 0, C2 = 256, C3 = 320, C4 = 352, C5 = 416, TMEM_COLS = 512;

constexpr uint32_t ID_N16 = tc::idesc_bf16(128, 16);
constexpr uint32_t ID_N32 = tc::idesc_bf16(128, 32);
constexpr uint32_t ID_N64 = tc::idesc_bf16(128, 64);
constexpr int kMaxPolls = 1 << 22;   // non-suspending tests: tens of ms

__device__ __forceinline__ int boff(int n, int k, int lbo) {   // B element (n, k)
  return (k >> 3) * lbo + (n >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
}

// Weights into their operand layouts, biases, zeros in both phase-map regions
// (their border entries are never written again). Ends with a barrier.
__device__ __forceinline__ void stage(const void* packed_w, uint8_t* sm) {
  const net::Packed P = net::packed(packed_w);
  const int tid = threadIdx.x, nt = blockDim.x;
  uint4* z = reinterpret_cast<uint4*>(sm + H1_OFF);
  for (int i = tid; i < (BIAS_OFF - H1_OFF) / 16; i += nt) z[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int e = tid; e < 3 * 32 * 16; e += nt) {
    const int u = e >> 9, n = (e >> 4) & 31, k = e & 15;
    const int v = 2 * (k >> 3) + ((k & 7) >> 2), c = k & 3;
    const uint16_t w = v <= 2 ? P.w[net::OFF_W1 + n * net::K1 + c * 9 + u * 3 + v] : 0;
    *reinterpret_cast<uint16_t*>(sm + W1_OFF + u * 1024 + boff(n, k, 512)) = w;
  }
  for (int e = tid; e < 2 * 18 * 32 * 16; e += nt) {
    const int layer = e / (18 * 512), rem = e - layer * 18 * 512;
    const int th = rem >> 9, n = (rem >> 4) & 31, k = rem & 15;
    const int tap = th >> 1, h = th & 1;
    const int src = (layer ? net::OFF_W3 : net::OFF_W2) + n * net::K2 + (16 * h + k) * 9 + tap;
    *reinterpret_cast<uint16_t*>(sm + (layer ? W3_OFF : W2_OFF) + th * 1024 + boff(n, k, 512)) =
        P.w[src];
  }
  for (int e = tid; e < 64 * 128; e += nt) {
    const int n = e >> 7, kp = e & 127;          // kp = position * 32 + channel
    const int k = (kp & 31) * 4 + (kp >> 5);     // flatten index (channel, row, col)
    *reinterpret_cast<uint16_t*>(sm + W4_OFF + boff(n, kp, 1024)) =
        P.w[net::OFF_W4 + n * net::K4 + k];
  }
  for (int e = tid; e < 16 * 64; e += nt) {
    const int n = e >> 6, k = e & 63;
    *reinterpret_cast<uint16_t*>(sm + W5_OFF + boff(n, k, 256)) =
        n < net::N5 ? P.w[net::OFF_W5 + n * net::K5 + k] : (uint16_t)0;
  }
  float* b = reinterpret_cast<float*>(sm + BIAS_OFF);
  for (int i = tid; i < net::N_BIAS; i += nt) b[i] = P.b[i];
  __syncthreads();
}

// BF16 bits (high half of the result) of (byte k of w - 128) / 64, exact:
// 2^23 + byte as a float, scaled and shifted by one rounding-free FMA.
__device__ __forceinline__ uint32_t byte_bf(uint32_t w, uint32_t k) {
  const float f = __uint_as_float(__byte_perm(w, 0x4B00u, 0x5440u | k));
  return __float_as_uint(__fmaf_rn(f, 1.f / 64.f, -131074.f));
}

// Half H of the conv1 operand entries of input row r (0..15) of group sample
// s (entries q = 0..4, or 5..8, of pixel pairs X = 2q, 2q + 1 of the bordered
// row): lo[x] and hi[x] = the BF16 pairs (channels 0, 1) and (channels 2, 3)
// of pixel x, read for x = 2q - 1 and 2q inside 0..15 only.
template <int H>
__device__ __forceinline__ void store_row(uint8_t* sm, int s, int r, const uint32_t (&lo)[16],
                                          const uint32_t (&hi)[16]) {
  const int Y = r + 1, pu = Y & 1, a = Y >> 1;
  uint8_t* base = sm + P_OFF + pu * 2 * P_MAP + a * P_ROW + s * 16;
#pragma unroll
  for (int q = H ? 5 : 0; q < (H ? 9 : 5); ++q) {
    const uint4 e = make_uint4(q > 0 ? lo[2 * q - 1] : 0u, q > 0 ? hi[2 * q - 1] : 0u,
                               q < 8 ? lo[2 * q] : 0u, q < 8 ? hi[2 * q] : 0u);
    if (q <= 7) *reinterpret_cast<uint4*>(base + q * 128) = e;
    if (q >= 1) *reinterpret_cast<uint4*>(base + P_MAP + (q - 1) * 128) = e;
  }
}

// The zero top row (bordered row 0) of conv1's input: 128 entries, one per
// thread of the first 128 (the region also holds the fc operands between
// rounds).
__device__ __forceinline__ void store_top_rows(uint8_t* sm) {
  const int e = threadIdx.x;   // shift, col, sample
  if (e < 128)
    *reinterpret_cast<uint4*>(sm + P_OFF + (e >> 6) * P_MAP + (e & 63) * 16) =
        make_uint4(0u, 0u, 0u, 0u);
}

// This thread's input item: group sample s = tid % 8 (the 8 lanes of a store
// phase are 8 samples), row r = (tid / 8) % 16, and (with 8 epilogue warps)
// half of the row tid / 128, else the whole row.
__device__ __forceinline__ int item_sample() { return threadIdx.x & 7; }
__device__ __forceinline__ int item_row() { return (threadIdx.x >> 3) & 15; }

// Half H of row r of group sample s from four rows of 16 bytes (channels
// 0..3, pixels as bytes, 0x80 where outside the level).
template <int H>
__device__ __forceinline__ void store_row_bytes(uint8_t* sm, int s, int r,
                                                const uint32_t (&px)[4][4]) {
  uint32_t lo[16], hi[16];
#pragma unroll
  for (int x = H ? 9 : 0; x < (H ? 16 : 9); ++x) {
    const uint32_t k = (uint32_t)(x & 3);
    lo[x] = __byte_perm(byte_bf(px[0][x >> 2], k), byte_bf(px[1][x >> 2], k), 0x7632);
    hi[x] = __byte_perm(byte_bf(px[2][x >> 2], k), byte_bf(px[3][x >> 2], k), 0x7632);
  }
  store_row<H>(sm, s, r, lo, hi);
}

// Half H of row r of group sample s from BF16 rows: v[ch][k] = pixels 2k, 2k + 1.
template <int H>
__device__ __forceinline__ void store_row_bf16(uint8_t* sm, int s, int r,
                                               const uint32_t (&v)[4][8]) {
  uint32_t lo[16], hi[16];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    lo[2 * k] = __byte_perm(v[0][k], v[1][k], 0x5410);
    lo[2 * k + 1] = __byte_perm(v[0][k], v[1][k], 0x7632);
    hi[2 * k] = __byte_perm(v[2][k], v[3][k], 0x5410);
    hi[2 * k + 1] = __byte_perm(v[2][k], v[3][k], 0x7632);
  }
  store_row<H>(sm, s, r, lo, hi);
}

// CW (16 or 32) accumulator columns of this warp's lanes (tc::ld16 / ld32).
__device__ __forceinline__ void ld_cols(uint32_t ta, float (&v)[32]) { tc::ld32(ta, v); }
__device__ __forceinline__ void ld_cols(uint32_t ta, float (&v)[16]) { tc::ld16(ta, v); }

__device__ __forceinline__ uint32_t relu_bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(a, 0.f), fmaxf(b, 0.f));
  return *reinterpret_cast<const uint32_t*>(&h);
}

// NC chunks of 8 accumulator columns + bias, ReLU, BF16.
template <int NC>
__device__ __forceinline__ void act(const float* v, const float* bias, uint4 (&q)[NC]) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int n = 8 * c;
    q[c] = make_uint4(relu_bf2(v[n] + bias[n], v[n + 1] + bias[n + 1]),
                      relu_bf2(v[n + 2] + bias[n + 2], v[n + 3] + bias[n + 3]),
                      relu_bf2(v[n + 4] + bias[n + 4], v[n + 5] + bias[n + 5]),
                      relu_bf2(v[n + 6] + bias[n + 6], v[n + 7] + bias[n + 7]));
  }
}

// Writes chunks c0 .. c0 + NC - 1 (8 channels each) of pixel (Y, X)
// (bordered, interior) of a layer's output into the next layer's phase maps
// (COLS columns and NS samples per map row): odd X into the odd-column map,
// even X into the even-column map (when inside it) and the map shifted by
// one column.
template <int MAP, int CHUNK, int COLS, int NS, int NC>
__device__ __forceinline__ void store_phase(uint8_t* region, int Y, int X, int s, int c0,
                                            const uint4 (&q)[NC]) {
  const int half = X >> 1;
  uint8_t* row = region + (Y & 1) * 3 * MAP + (Y >> 1) * COLS * NS * 16 + s * 16 + c0 * CHUNK;
  auto put = [&](int var, int col) {
    uint8_t* p = row + var * MAP + col * NS * 16;
#pragma unroll
    for (int c = 0; c < NC; ++c) *reinterpret_cast<uint4*>(p + c * CHUNK) = q[c];
  };
  if (X & 1) {
    put(1, half);
  } else {
    if (half < COLS) put(0, half);
    put(2, half - 1);
  }
}

// mbarriers: completions of the MMAs (conv1 and conv2 by group parity, the
// per-round layers) and operands ready (one arrival per epilogue warp).
enum Bar { B_C1 = 0, B_C2 = 2, B_R = 4, B_P = 5, B_H1 = 6, B_H2 = 7, B_H3 = 8, B_H4 = 9 };

// Runs every round of a source on this CTA (rounds blockIdx.x, + gridDim.x,
// ...). Src provides: Tile, Regs; n_tiles(); tile(v) (its sample count nv);
// load(tile, g, regs): this thread's input item of group g into registers
// (item_sample(), item_row()); store(sm, regs): that item into conv1's
// operand; write(tile, s, dx, dy, conf). THREADS threads.
//
// Warp-specialised: warp EPI_WARPS only issues MMAs, each layer as soon as
// its operand is complete (an mbarrier that every epilogue warp arrives on);
// the epilogue warps stage inputs and drain the accumulators, waiting only on
// MMA completions. Warp w < EPI_WARPS reads the accumulator lanes of quarter
// w % 4 and (with 8 epilogue warps) its half w / 4 of the columns (or of
// conv1's tiles). conv1 and
// conv2 accumulate into buffers chosen by group parity, so that in step g the
// tensor core runs conv1(g + 1) and conv2(g) while the epilogue warps drain
// conv1(g) and conv2(g - 1):
//   epilogue: wait conv1(g) | store input g + 1 -> ready | wait conv2(g - 1) |
//             drain conv1(g) -> ready | drain conv2(g - 1)
//   issuer:   wait ready -> conv1(g + 1) | wait ready -> conv2(g)
// (an MMA of 128 rows x 16 K costs about 50-65 cycles to issue, the tensor
// core's reading of its 4-5 KB of operands, and completes shortly after the
// last one is issued).
// Every wait is bounded; one that gives up sets a shared abort flag, which
// every other wait also stops on, then the kernel records VIO_ERR_TIMEOUT in
// *fault (when not null), lets the MMAs in flight finish (bounded) and frees
// its tensor memory.
template <class Src>
__device__ __forceinline__ void run(const Src& src, const void* packed_w, uint8_t* sm,
                                    int32_t* fault) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = 32 * (warp & 3), hw = NH > 1 ? (warp >> 2) & 1 : 0;
  const int n_tiles = src.n_tiles();
  if ((int)blockIdx.x >= n_tiles) return;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + BAR_OFF);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + SLOT_OFF);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + SLOT_OFF + 4);
  const bool issuer = warp == EPI_WARPS;
  typename Src::Regs R;
  int v = blockIdx.x;
  typename Src::Tile cur = src.tile(v), nxt = cur;
  if (!issuer) src.load(cur, 0, R);
  stage(packed_w, sm);
  if (tid == 0) {
    for (int b = 0; b < N_BARS; ++b) tc::mbar_init(bar + b, b < B_P ? 1 : EPI_WARPS);
    tc::fence_mbar_init();
    *abort_flag = 0;
  }
  if (warp == 0) tc::tmem_alloc(slot, TMEM_COLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tm = *slot;
  const uint32_t sb = tc::smem_u32(sm);
  const float* bias = reinterpret_cast<const float*>(sm + BIAS_OFF);
  uint32_t ph = 0;    // phase bits of the barriers this thread waits on (bit b)
  // bounded wait for the next phase of barrier b; false on a time-out or abort
  auto wait = [&](int b) -> bool {
    const uint32_t parity = (ph >> b) & 1u;
    for (int i = 0; i < kMaxPolls; ++i) {
      if (tc::mbar_try(bar + b, parity)) {
        ph ^= 1u << b;
        tc::fence_after();
        return true;
      }
      if ((i & 63) == 63 && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
  };
  // an epilogue warp's operand writes made visible to the tensor core, then
  // its arrival on ready barrier b
  auto ready = [&](int b) {
    tc::fence_smem_to_async();
    tc::fence_before();
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(bar + b);
  };

  if (issuer) {
    // Descriptors: a layer's base descriptor plus the operand's byte offset /
    // 16 (the start address field is the low bits; every address stays below
    // 256 KB), the offsets compile-time constants of the unrolled loops.
    const uint64_t dP = tc::sdesc(sb + P_OFF, P_MAP, 128);
    const uint64_t dH1 = tc::sdesc(sb + H1_OFF, H1_CHUNK, 128);
    const uint64_t dH2 = tc::sdesc(sb + H2_OFF, H2_CHUNK, 128);
    const uint64_t dH3 = tc::sdesc(sb + H3_OFF, 512, 128);
    const uint64_t dH4 = tc::sdesc(sb + H4_OFF, 512, 128);
    const uint64_t dW1 = tc::sdesc(sb + W1_OFF, 512, 128);
    const uint64_t dW2 = tc::sdesc(sb + W2_OFF, 512, 128);
    const uint64_t dW3 = tc::sdesc(sb + W3_OFF, 512, 128);
    const uint64_t dW4 = tc::sdesc(sb + W4_OFF, 1024, 128);
    const uint64_t dW5 = tc::sdesc(sb + W5_OFF, 256, 128);
    // conv2 and conv3: 9 taps x 2 K halves over the phase maps of their input
    auto conv3x3 = [&](uint32_t d, uint64_t dA, int map, int chunk, int row, uint64_t dB) {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int u = tap / 3, m = (u & 1) * 3 + tap % 3;
          tc::mma_bf16(d, dA + ((m * map + 2 * h * chunk + (u >> 1) * row) >> 4),
                       dB + (((2 * tap + h) * 1024) >> 4), ID_N32, (tap | h) != 0);
        }
    };
    auto conv1 = [&](int g) {
      if (lane == 0) {
        const uint32_t d = tm + C1 + 128 * (g & 1);
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
          for (int t = 0; t < 4; ++t)
            tc::mma_bf16(d + 32 * t,
                         dP + (((u & 1) * 2 * P_MAP + (2 * t + (u >> 1)) * P_ROW) >> 4),
                         dW1 + ((u * 1024) >> 4), ID_N32, u > 0);
        tc::commit(bar + B_C1 + (g & 1));
      }
      __syncwarp();
    };
    for (; v < n_tiles && !*abort_flag; v += gridDim.x) {
      const int ng = (src.tile(v).nv + GROUP - 1) / GROUP;
      // the epilogue warps' order: input g + 1 is ready before conv1(g)'s
      // output has been drained, so conv1(g + 1) goes ahead of conv2(g)
      bool ok = wait(B_P);
      if (ok) conv1(0);
      for (int g = 0; g < ng && ok; ++g) {
        if (g + 1 < ng) {
          if (!(ok = wait(B_P))) break;
          conv1(g + 1);
        }
        if (!(ok = wait(B_H1))) break;
        if (lane == 0) {
          conv3x3(tm + C2 + 32 * (g & 1), dH1, H1_MAP, H1_CHUNK, 512, dW2);
          tc::commit(bar + B_C2 + (g & 1));
        }
        __syncwarp();
      }
      if (!ok || !wait(B_H2)) break;
      if (lane == 0) {
        conv3x3(tm + C3, dH2, H2_MAP, H2_CHUNK, 1024, dW3);
        tc::commit(bar + B_R);
      }
      __syncwarp();
      if (!wait(B_H3)) break;
      if (lane == 0) {
#pragma unroll
        for (int h = 0; h < 8; ++h)
          tc::mma_bf16(tm + C4, dH3 + ((2 * h * 512) >> 4), dW4 + ((2 * h * 1024) >> 4), ID_N64,
                       h > 0);
        tc::commit(bar + B_R);
      }
      __syncwarp();
      if (!wait(B_H4)) break;
      if (lane == 0) {
#pragma unroll
        for (int h = 0; h < 4; ++h)
          tc::mma_bf16(tm + C5, dH4 + ((2 * h * 512) >> 4), dW5 + ((2 * h * 256) >> 4), ID_N16,
                       h > 0);
        tc::commit(bar + B_R);
      }
      __syncwarp();
    }
  } else {
    // conv1's epilogue of group g: this warp's two tiles; row = (position p
    // of output rows 2t, 2t + 1, sample) -> conv2's phase maps
    auto epi1 = [&](int g) {
      constexpr int TW = 4 / NH;   // tiles per warp
      const int col = C1 + 128 * (g & 1) + 32 * TW * hw;
      const int r = quarter + lane, p = r >> 3;
#pragma unroll 1
      for (int k = 0; k < TW; ++k) {
        float f[32];
        tc::ld32(tc::taddr(tm, quarter, col + 32 * k), f);
        uint4 q[4];
        act<4>(f, bias + net::OFF_B1, q);
        store_phase<H1_MAP, H1_CHUNK, 4, GROUP, 4>(
            sm + H1_OFF, 2 * (TW * hw + k) + (p >> 3) + 1, (p & 7) + 1, r & 7, 0, q);
      }
    };
    // conv2's epilogue of group g: row (position p, sample), this warp's 16
    // channels -> conv3's phase maps
    auto epi2 = [&](int g) {
      constexpr int CW = 32 / NH, NC = CW / 8;   // columns, chunks per warp
      const int r = quarter + lane, p = r >> 3;
      float a[CW];
      uint4 q[NC];
      ld_cols(tc::taddr(tm, quarter, C2 + 32 * (g & 1) + CW * hw), a);
      act<NC>(a, bias + net::OFF_B2 + CW * hw, q);
      store_phase<H2_MAP, H2_CHUNK, 2, ROUND, NC>(sm + H2_OFF, (p >> 2) + 1, (p & 3) + 1,
                                                  GROUP * g + (r & 7), NC * hw, q);
    };
    for (;;) {
      const int ng = (cur.nv + GROUP - 1) / GROUP;
      const int v_next = v + (int)gridDim.x;
      // the next input after group g's: this tile's group g + 1, else the
      // next tile's first
      auto prefetch_after = [&](int g) {
        if (g + 1 < ng) {
          src.load(cur, g + 1, R);
        } else if (v_next < n_tiles) {
          nxt = src.tile(v_next);
          src.load(nxt, 0, R);
        }
      };
      src.store(sm, R);
      store_top_rows(sm);
      ready(B_P);
      prefetch_after(0);
      bool ok = true;
      for (int g = 0; g < ng && ok; ++g) {
        if (!(ok = wait(B_C1 + (g & 1)))) break;              // conv1(g): its input is free
        if (g + 1 < ng) {
          src.store(sm, R);
          ready(B_P);
          prefetch_after(g + 1);
        }
        if (g > 0 && !(ok = wait(B_C2 + ((g - 1) & 1)))) break;   // conv2(g - 1) done
        epi1(g);
        ready(B_H1);
        if (g > 0) epi2(g - 1);
      }
      if (!ok || !wait(B_C2 + ((ng - 1) & 1))) break;
      epi2(ng - 1);
      ready(B_H2);
      if (!wait(B_R)) break;
      {   // conv3 epilogue: row = (position warp % 4, sample lane), this warp's
          // channels -> fc1 input at K = position * 32 + channel
        constexpr int CW = 32 / NH, NC = CW / 8;
        float a[CW];
        uint4 q[NC];
        ld_cols(tc::taddr(tm, quarter, C3 + CW * hw), a);
        act<NC>(a, bias + net::OFF_B3 + CW * hw, q);
        uint8_t* o = sm + H3_OFF + (lane >> 3) * 128 + (lane & 7) * 16;
#pragma unroll
        for (int c = 0; c < NC; ++c)
          *reinterpret_cast<uint4*>(o + (4 * (warp & 3) + NC * hw + c) * 512) = q[c];
      }
      ready(B_H3);
      if (!wait(B_R)) break;
      if (quarter == 0) {   // fc1 epilogue: rows 0..31 = the samples, 64 / NH columns per warp
        uint8_t* o = sm + H4_OFF + (lane >> 3) * 128 + (lane & 7) * 16;
#pragma unroll 1
        for (int half = hw; half < 2; half += NH) {
          float a[32];
          uint4 q[4];
          tc::ld32(tc::taddr(tm, 0, C4 + 32 * half), a);
          act<4>(a, bias + net::OFF_B4 + 32 * half, q);
#pragma unroll
          for (int c = 0; c < 4; ++c) *reinterpret_cast<uint4*>(o + (4 * half + c) * 512) = q[c];
        }
      }
      ready(B_H4);
      if (!wait(B_R)) break;
      if (warp == 0) {
        float a[16];
        tc::ld16(tc::taddr(tm, 0, C5), a);
        if (lane < cur.nv) {
          const float o0 = a[0] + bias[net::OFF_B5], o1 = a[1] + bias[net::OFF_B5 + 1];
          const float o2 = a[2] + bias[net::OFF_B5 + 2];
          src.write(cur, lane, o0 * net::kScale, o1 * net::kScale, 1.f / (1.f + expf(-o2)));
        }
      }
      if (v_next >= n_tiles) break;
      cur = nxt;
      v = v_next;
    }
  }
  __syncthreads();
  if (*abort_flag) {
    // every MMA issued before a further commit has completed when it arrives
    if (tid == 32 * EPI_WARPS) {
      if (fault) atomicExch(fault, (int32_t)VIO_ERR_TIMEOUT);
      tc::mbar_init(bar + B_P, 1);
      tc::commit(bar + B_P);
      tc::mbar_wait(bar + B_P, 0, kMaxPolls);
    }
    __syncthreads();
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tm, TMEM_COLS);
}

// Source of rounds: inputs [n][4][16][16] BF16 in global memory, outputs
// [n][3] (dx, dy, conf).
struct XSource {
  const uint16_t* x;
  int n;
  float* out;
  struct Tile {
    int s0, nv;
  };
  struct Regs {
    uint32_t v[4][8];
  };
  __device__ int n_tiles() const { return (n + ROUND - 1) / ROUND; }
  __device__ Tile tile(int t) const { return Tile{t * ROUND, min(ROUND, n - t * ROUND)}; }
  __device__ void load(const Tile& T, int g, Regs& R) const {
    const int i = g * GROUP + item_sample(), r = item_row();
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
      uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
      if (i < T.nv) {
        const uint4* p =
            reinterpret_cast<const uint4*>(x + (long long)(T.s0 + i) * 1024 + ch * 256 + r * 16);
        lo = __ldg(p);
        hi = __ldg(p + 1);
      }
      R.v[ch][0] = lo.x;
      R.v[ch][1] = lo.y;
      R.v[ch][2] = lo.z;
      R.v[ch][3] = lo.w;
      R.v[ch][4] = hi.x;
      R.v[ch][5] = hi.y;
      R.v[ch][6] = hi.z;
      R.v[ch][7] = hi.w;
    }
  }
  __device__ void store(uint8_t* sm, const Regs& R) const {
    if (NH == 1 || (threadIdx.x >> 7)) store_row_bf16<1>(sm, item_sample(), item_row(), R.v);
    if (NH == 1 || !(threadIdx.x >> 7)) store_row_bf16<0>(sm, item_sample(), item_row(), R.v);
  }
  __device__ void write(const Tile& T, int s, float dx, float dy, float conf) const {
    float* o = out + 3LL * (T.s0 + s);
    o[0] = dx;
    o[1] = dy;
    o[2] = conf;
  }
};

// The 16 bytes of a prefetched input row (net::RowWords), aligned to its
// first pixel, 0x80 (input 0) where the pixel lies outside the level.
__device__ __forceinline__ void row_bytes(const net::RowWords& R, uint32_t (&b)[4]) {
  const unsigned sh = 8u * (unsigned)(R.cx - R.x4);
  const int valid = R.wl - R.cx;   // pixels inside the level from the first
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t a = __funnelshift_r(R.w[k], R.w[k + 1], sh);
    const int vk = valid - 4 * k;
    const uint32_t keep = vk >= 4 ? 0xffffffffu : (vk <= 0 ? 0u : (1u << (8 * vk)) - 1u);
    b[k] = (a & keep) | (0x80808080u & ~keep);
  }
}

}  // namespace ntc
}  // namespace vio
