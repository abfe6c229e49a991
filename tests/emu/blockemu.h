// Host emulation of CUDA thread blocks, for running the library's device code
// on the CPU under AddressSanitizer (test infrastructure). One std::thread per
// CUDA thread; __syncthreads, named barriers and the warp collectives
// (__ballot_sync, __shfl*_sync, __reduce_max_sync, __syncwarp) are barriers
// over the threads that must all reach them, so code that calls a full-mask
// collective from divergent lanes stops with "EMU DEADLOCK" instead of
// hanging; __syncthreads_or too. Integer and bit intrinsics (__byte_perm,
// __vminu2, __vmaxu2, __popc, __ffs, __funnelshift_r, __fmaf_rn, atomicMax,
// atomicExch, atomicAdd) are plain host functions, as are the tracker's float
// intrinsics (__fmul_rn, __fadd_rd, rsqrtf, __fdividef).
#pragma once
#include <cuda_runtime.h>
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

struct EmuDim { unsigned x = 0, y = 0, z = 0; };
static thread_local EmuDim threadIdx;
static EmuDim blockDim{128, 1, 1};
static thread_local EmuDim blockIdx;
static EmuDim gridDim{1, 1, 1};

struct EmuBarrier {
  std::mutex m; std::condition_variable cv; int n, count = 0; long gen = 0;
  explicit EmuBarrier(int n_) : n(n_) {}
  void wait() {
    std::unique_lock<std::mutex> l(m);
    long g = gen;
    if (++count == n) { count = 0; ++gen; cv.notify_all(); return; }
    if (!cv.wait_for(l, std::chrono::seconds(20), [&] { return gen != g; })) {
      fprintf(stderr, "EMU DEADLOCK (barrier of %d, %d arrived)\n", n, count); std::abort();
    }
  }
};
struct EmuWarp { EmuBarrier bar{32}; uint64_t vals[32]; };
struct EmuBlock {
  EmuBarrier block_bar;
  std::vector<std::unique_ptr<EmuWarp>> warps;
  std::mutex nm; std::map<int, std::unique_ptr<EmuBarrier>> named;
  int or_acc[3] = {0, 0, 0};   // __syncthreads_or, rounds in turn
  explicit EmuBlock(int nt) : block_bar(nt) { for (int i = 0; i < nt / 32; ++i) warps.emplace_back(new EmuWarp); }
};
static thread_local EmuBlock* emu_blk = nullptr;
inline EmuWarp& emu_warp() { return *emu_blk->warps[threadIdx.x >> 5]; }
inline void __syncthreads() { emu_blk->block_bar.wait(); }
inline void __syncwarp(unsigned = 0xffffffffu) { emu_warp().bar.wait(); }
static thread_local int emu_or_round = 0;
// Round k ORs into slot k % 3; after its barrier thread 0 clears the slot of
// round k + 2, which no thread can reach before the barrier of round k + 1.
inline int __syncthreads_or(int p) {
  const int k = emu_or_round++ % 3;
  { std::lock_guard<std::mutex> l(emu_blk->nm); emu_blk->or_acc[k] |= (p != 0); }
  __syncthreads();
  int r;
  { std::lock_guard<std::mutex> l(emu_blk->nm); r = emu_blk->or_acc[k];
    if (threadIdx.x == 0) emu_blk->or_acc[(k + 2) % 3] = 0; }
  return r;
}
inline void emu_bar(int id, int n) {
  EmuBarrier* b;
  { std::lock_guard<std::mutex> l(emu_blk->nm);
    auto& p = emu_blk->named[id];
    if (!p) p.reset(new EmuBarrier(n));
    if (p->n != n) { fprintf(stderr, "named barrier count mismatch\n"); std::abort(); }
    b = p.get(); }
  b->wait();
}
template <class F> inline uint64_t emu_collect(uint64_t v, F f) {
  auto& w = emu_warp(); int lane = threadIdx.x & 31;
  w.vals[lane] = v; w.bar.wait(); uint64_t r = f(w.vals, lane); w.bar.wait(); return r;
}
inline void emu_check_full(unsigned mask) { if (mask != 0xffffffffu) { fprintf(stderr, "partial mask\n"); std::abort(); } }
inline unsigned __ballot_sync(unsigned mask, int p) {
  emu_check_full(mask);
  return (unsigned)emu_collect(p != 0, [](uint64_t* v, int) { unsigned r = 0; for (int i = 0; i < 32; ++i) if (v[i]) r |= 1u << i; return (uint64_t)r; });
}
inline int __any_sync(unsigned mask, int p) { return __ballot_sync(mask, p) != 0; }
template <class T> inline T __shfl_sync(unsigned mask, T v, int src) {
  emu_check_full(mask); uint64_t u = 0; memcpy(&u, &v, sizeof(T));
  uint64_t r = emu_collect(u, [src](uint64_t* vv, int) { return vv[src & 31]; });
  T o; memcpy(&o, &r, sizeof(T)); return o;
}
template <class T> inline T __shfl_up_sync(unsigned mask, T v, int d) {
  emu_check_full(mask); uint64_t u = 0; memcpy(&u, &v, sizeof(T));
  uint64_t r = emu_collect(u, [d](uint64_t* vv, int lane) { return lane >= d ? vv[lane - d] : vv[lane]; });
  T o; memcpy(&o, &r, sizeof(T)); return o;
}
template <class T> inline T __shfl_xor_sync(unsigned mask, T v, int d) {
  emu_check_full(mask); uint64_t u = 0; memcpy(&u, &v, sizeof(T));
  uint64_t r = emu_collect(u, [d](uint64_t* vv, int lane) { return vv[lane ^ d]; });
  T o; memcpy(&o, &r, sizeof(T)); return o;
}
template <class T> inline T __shfl_down_sync(unsigned mask, T v, int d) {
  emu_check_full(mask); uint64_t u = 0; memcpy(&u, &v, sizeof(T));
  uint64_t r = emu_collect(u, [d](uint64_t* vv, int lane) { return lane + d < 32 ? vv[lane + d] : vv[lane]; });
  T o; memcpy(&o, &r, sizeof(T)); return o;
}
inline unsigned __reduce_max_sync(unsigned mask, unsigned v) {
  emu_check_full(mask);
  return (unsigned)emu_collect(v, [](uint64_t* vv, int) { uint64_t m = 0; for (int i = 0; i < 32; ++i) m = std::max(m, vv[i]); return m; });
}
inline int __popc(unsigned v) { return __builtin_popcount(v); }
inline int __popcll(unsigned long long v) { return __builtin_popcountll(v); }
inline int __ffs(unsigned v) { return __builtin_ffs((int)v); }
inline int __clz(unsigned v) { return v ? __builtin_clz(v) : 32; }
inline unsigned __byte_perm(unsigned x, unsigned y, unsigned s) {
  uint8_t b[8];
  for (int i = 0; i < 4; ++i) { b[i] = (x >> (8 * i)) & 0xff; b[4 + i] = (y >> (8 * i)) & 0xff; }
  unsigned r = 0;
  for (int i = 0; i < 4; ++i) r |= (unsigned)b[(s >> (4 * i)) & 7] << (8 * i);
  return r;
}
inline unsigned __vminu2(unsigned a, unsigned b) {
  unsigned lo = std::min(a & 0xffffu, b & 0xffffu), hi = std::min(a >> 16, b >> 16); return lo | (hi << 16); }
inline unsigned __vmaxu2(unsigned a, unsigned b) {
  unsigned lo = std::max(a & 0xffffu, b & 0xffffu), hi = std::max(a >> 16, b >> 16); return lo | (hi << 16); }
template <class T> inline T __ldg(const T* p) { return *p; }
inline float __uint_as_float(unsigned u) { float f; memcpy(&f, &u, 4); return f; }
inline float __int_as_float(int u) { float f; memcpy(&f, &u, 4); return f; }
inline unsigned __float_as_uint(float f) { unsigned u; memcpy(&u, &f, 4); return u; }
inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
inline float __fmul_rn(float a, float b) { return a * b; }
inline int __float_as_int(float f) { int u; memcpy(&u, &f, 4); return u; }
// a + b rounded toward -inf: the nearest sum, stepped down when the exact
// rounding error (TwoSum) shows it above the exact sum
inline float __fadd_rd(float a, float b) {
  const float s = a + b, bb = s - a;
  const float err = (a - (s - bb)) + (b - bb);
  return err < 0.f ? std::nextafter(s, -INFINITY) : s;
}
inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
inline float __fdividef(float a, float b) { return a / b; }
inline unsigned __funnelshift_r(unsigned lo, unsigned hi, unsigned sh) {
  sh &= 31; return sh ? (lo >> sh) | (hi << (32 - sh)) : lo; }
inline size_t __cvta_generic_to_shared(const void*) { fprintf(stderr, "cvta on the host\n"); std::abort(); }
using std::min; using std::max;
inline int min(int a, int b) { return a < b ? a : b; }
inline int max(int a, int b) { return a > b ? a : b; }
inline unsigned min(unsigned a, unsigned b) { return a < b ? a : b; }
inline unsigned max(unsigned a, unsigned b) { return a > b ? a : b; }
inline long long min(long long a, long long b) { return a < b ? a : b; }
inline long long max(long long a, long long b) { return a > b ? a : b; }

// runs body(tid) for every thread of one block
inline void emu_run_block(int nt, const std::function<void()>& body, EmuDim bidx) {
  blockDim.x = nt;
  EmuBlock blk(nt);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] { emu_blk = &blk; threadIdx.x = t; blockIdx = bidx; body(); });
  for (auto& x : th) x.join();
}
static std::mutex emu_atomic_mu;
inline int atomicAdd(int* p, int v) { std::lock_guard<std::mutex> l(emu_atomic_mu); int o = *p; *p += v; return o; }
inline float atomicAdd(float* p, float v) { std::lock_guard<std::mutex> l(emu_atomic_mu); float o = *p; *p += v; return o; }

// mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 of one warp, with the
// fragment layout of the PTX ISA (groupID g = lane / 4, t = lane % 4):
// A (16 x 16, row-major) a[0]: (g, 2t..2t+1), a[1]: (g+8, 2t..), a[2]:
// (g, 2t+8..), a[3]: (g+8, 2t+8..); B (16 x 8) b0: rows 2t..2t+1 of column g,
// b1: rows 2t+8..2t+9; C and D c0, c1: (g, 2t..2t+1), c2, c3: (g+8, 2t..);
// the lower half of a 32-bit register holds the lower column (row of B).
// Every lane posts its fragments, then computes its own four outputs.
struct EmuMma { uint32_t a[32][4]; uint32_t b[32][2]; };
inline EmuMma& emu_mma_buf() {
  static std::mutex m;
  static std::map<const void*, std::unique_ptr<EmuMma>> bufs;
  std::lock_guard<std::mutex> l(m);
  auto& p = bufs[&emu_warp()];
  if (!p) p.reset(new EmuMma);
  return *p;
}
inline float emu_bf16_bits(uint32_t w, int hi) {
  const uint32_t u = (hi ? (w >> 16) : (w & 0xffffu)) << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}
inline void emu_mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  EmuMma& M = emu_mma_buf();
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < 4; ++i) M.a[lane][i] = a[i];
  M.b[lane][0] = b0;
  M.b[lane][1] = b1;
  emu_warp().bar.wait();
  auto A = [&](int r, int k) {
    return emu_bf16_bits(M.a[(r & 7) * 4 + ((k & 7) >> 1)][(r >> 3) + 2 * (k >> 3)], k & 1);
  };
  auto B = [&](int k, int n) {
    return emu_bf16_bits(M.b[n * 4 + ((k & 7) >> 1)][k >> 3], k & 1);
  };
  const int g = lane >> 2, t = lane & 3;
  float out[4];
  for (int e = 0; e < 4; ++e) {
    const int r = g + 8 * (e >> 1), n = 2 * t + (e & 1);
    float s = 0.f;
    for (int k = 0; k < 16; ++k) s += A(r, k) * B(k, n);
    out[e] = d[e] + s;
  }
  emu_warp().bar.wait();       // every lane has read the fragments
  for (int e = 0; e < 4; ++e) d[e] = out[e];
}
inline int atomicExch(int* p, int v) { std::lock_guard<std::mutex> l(emu_atomic_mu); int o = *p; *p = v; return o; }
inline unsigned long long atomicMax(unsigned long long* p, unsigned long long v) {
  std::lock_guard<std::mutex> l(emu_atomic_mu); unsigned long long o = *p; if (v > o) *p = v; return o; }
