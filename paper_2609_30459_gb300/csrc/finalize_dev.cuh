// Device code of the finalisation (K3 of frame.cu): one CTA of K3_THREADS
// threads per stream keeps the tracks that passed, counts them per cell,
// selects per cell the first k - count candidates (Sec. III-D with the cell
// buffer), appends them to camera 0 and their successful stereo matches to
// camera 1, and writes the counts and per-step statistics.
#pragma once
#include "frame.cuh"

namespace vio {

constexpr int K3_THREADS = 1024;

// Block-wide exclusive scan (one value per thread); returns the exclusive
// prefix and the block total. All threads must call it.
template <typename T>
__device__ __forceinline__ T block_scan(T v, T* warp_sums, T& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    T ws = lane < K3_THREADS / 32 ? warp_sums[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T t = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += t;
    }
    if (lane < K3_THREADS / 32) warp_sums[lane] = ws;
  }
  __syncthreads();
  total = warp_sums[K3_THREADS / 32 - 1];
  return (warp ? warp_sums[warp - 1] : T(0)) + incl - v;
}

__device__ __forceinline__ int cell_of(float x, int cw) {
  int c = (int)floorf(x / (float)cw);
  if ((float)(c + 1) * (float)cw <= x) ++c;
  if ((float)c * (float)cw > x) --c;
  return c;
}

constexpr int kRunMax = 16;   // slots (or cells) one thread owns in one pass

// Two block-wide exclusive scans sharing their two barriers (as block_scan).
__device__ __forceinline__ void block_scan2(unsigned a, unsigned long long b, unsigned* wa,
                                           unsigned long long* wb, unsigned& ea,
                                           unsigned long long& eb, unsigned& ta,
                                           unsigned long long& tb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned ia = a;
  unsigned long long ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned x = __shfl_up_sync(0xffffffffu, ia, o);
    const unsigned long long y = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) {
      ia += x;
      ib += y;
    }
  }
  if (lane == 31) {
    wa[warp] = ia;
    wb[warp] = ib;
  }
  __syncthreads();
  if (warp == 0) {
    unsigned x = lane < K3_THREADS / 32 ? wa[lane] : 0u;
    unsigned long long y = lane < K3_THREADS / 32 ? wb[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned u = __shfl_up_sync(0xffffffffu, x, o);
      const unsigned long long w = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) {
        x += u;
        y += w;
      }
    }
    if (lane < K3_THREADS / 32) {
      wa[lane] = x;
      wb[lane] = y;
    }
  }
  __syncthreads();
  ta = wa[K3_THREADS / 32 - 1];
  tb = wb[K3_THREADS / 32 - 1];
  ea = (warp ? wa[warp - 1] : 0u) + ia - a;
  eb = (warp ? wb[warp - 1] : 0ull) + ib - b;
}

// The finalisation in one pass, when the capacity and the cell count are at
// most K3_THREADS (thread t owns list slot t and cell t). Every global load
// the pass needs is issued at entry, so that their latencies overlap: the
// counts, the statuses, positions and ids of the owned slots, the owned
// cell's candidate count and its first candidate with its stereo match (the
// further candidates of a cell, k > 1, are read where used). Then the
// occupancy of the surviving camera-0 tracks is counted, the survivors' scan
// and the cells' selection scan run together (one pair of barriers), and
// every output is written from registers. Same lists, order and statistics
// as the phased version below.
__device__ __forceinline__ void finalize_one_pass(const FrameLaunch& f, int s, const StreamRef& sr,
                                                  int32_t* st, int* occ_s, unsigned* wsa,
                                                  unsigned long long* wsb) {
  __shared__ int learned_s;
  const int t = threadIdx.x;
  const int k = f.p.k_per_cell;
  const int gx = f.g.w[0] / f.p.cell_w, gy = f.g.h[0] / f.p.cell_h;
  const int n_cells = gx * gy;
  const int W = f.g.w[0];
  const long long cap = f.cap;
  const long long cbase = (long long)s * n_cells;
  const long long in0 = (((long long)sr.li * f.n_streams + s) * 2) * cap;
  const long long out0 = (((long long)sr.lo * f.n_streams + s) * 2) * cap;
  const long long trk0 = (2LL * s) * cap;
  const long long cnt_in = ((long long)sr.li * f.n_streams + s) * 2;
  const long long cnt_out = ((long long)sr.lo * f.n_streams + s) * 2;
  const bool slot_ok = t < f.cap, cell_ok = t < n_cells;
  // every load of the pass
  const int n0r = f.list_count[cnt_in], n1r = f.list_count[cnt_in + 1];
  const int id0 = f.next_id[s];
  int st0 = VIO_TRACK_EMPTY, st1 = VIO_TRACK_EMPTY, lid0 = 0, lid1 = 0, lr0 = 0, lr1 = 0;
  float x0 = 0.f, y0 = 0.f, x1 = 0.f, y1 = 0.f;
  if (slot_ok) {
    st0 = f.trk_status[trk0 + t];
    st1 = f.trk_status[trk0 + cap + t];
    x0 = f.trk_xy[2 * (trk0 + t)];
    y0 = f.trk_xy[2 * (trk0 + t) + 1];
    x1 = f.trk_xy[2 * (trk0 + cap + t)];
    y1 = f.trk_xy[2 * (trk0 + cap + t) + 1];
    lid0 = f.list_id[in0 + t];
    lid1 = f.list_id[in0 + cap + t];
    if (f.net) {
      lr0 = f.trk_learned[trk0 + t];
      lr1 = f.trk_learned[trk0 + cap + t];
    }
  }
  const long long q0 = (cbase + t) * k;   // the owned cell's first candidate
  int nc = 0, ss0 = VIO_TRACK_EMPTY;
  unsigned long long key0 = 0;
  float sx0 = 0.f, sy0 = 0.f;
  if (cell_ok) {
    nc = f.cand_count[cbase + t];
    key0 = f.cand[q0];
    if (!f.stereo_after) {
      ss0 = f.spec_status[q0];
      sx0 = f.spec_xy[2 * q0];
      sy0 = f.spec_xy[2 * q0 + 1];
    }
    occ_s[t] = 0;
  }
  if (t == 0) learned_s = 0;
  __syncthreads();

  // survivors of both cameras; occupancy of camera 0's
  const int n0 = sr.have_prev ? min(n0r, f.cap) : 0;
  const int n1 = sr.have_prev ? min(n1r, f.cap) : 0;
  const bool keep0 = t < n0 && st0 == VIO_TRACK_OK, keep1 = t < n1 && st1 == VIO_TRACK_OK;
  if (keep0 && x0 >= 0.f && y0 >= 0.f) {
    const int cx = cell_of(x0, f.p.cell_w), cy = cell_of(y0, f.p.cell_h);
    if (cx < gx && cy < gy) atomicAdd(&occ_s[cy * gx + cx], 1);
  }
  if (f.net) {
    const int nl = (keep0 ? lr0 : 0) + (keep1 ? lr1 : 0);
    if (nl) atomicAdd(&learned_s, nl);
  }
  __syncthreads();   // occupancy complete

  // the owned cell: selection (k_eff = k - occupancy), matched subset
  int nsel = 0, nm = 0;
  if (cell_ok) {
    const int occ = min(occ_s[t], 255);
    f.occupancy[cbase + t] = (uint8_t)occ;
    nsel = max(0, min(k - occ, nc));
    if (!f.stereo_after)
      for (int r = 0; r < nsel; ++r)
        nm += (r == 0 ? ss0 : (int)f.spec_status[q0 + r]) == VIO_TRACK_OK;
  }
  const unsigned long long packed = (unsigned long long)nsel | ((unsigned long long)nm << 21) |
                                    ((unsigned long long)nc << 42);
  unsigned sex, stot;
  unsigned long long cex, ctot;
  block_scan2((keep0 ? 1u : 0u) | (keep1 ? 0x10000u : 0u), packed, wsa, wsb, sex, cex, stot,
              ctot);
  const int surv0 = (int)(stot & 0xffffu), surv1 = (int)(stot >> 16);
  const int new_tot = (int)(ctot & 0x1fffff), m_tot = (int)((ctot >> 21) & 0x1fffff);
  const int c_tot = (int)((ctot >> 42) & 0x1fffff);

  // survivors, in order
  if (keep0) {
    const long long d = out0 + (sex & 0xffffu);
    f.list_xy[2 * d] = x0;
    f.list_xy[2 * d + 1] = y0;
    f.list_id[d] = lid0;
  }
  if (keep1) {
    const long long d = out0 + cap + (sex >> 16);
    f.list_xy[2 * d] = x1;
    f.list_xy[2 * d + 1] = y1;
    f.list_id[d] = lid1;
  }
  // the selected candidates: new keypoints, camera 0's list, camera 1's
  // successful matches
  const long long bn = (long long)s * cap;
  int o = (int)(cex & 0x1fffff), om = (int)((cex >> 21) & 0x1fffff);
  for (int r = 0; r < nsel; ++r, ++o) {
    const long long q = q0 + r;
    const unsigned idx = ~(unsigned)((r == 0 ? key0 : f.cand[q]) & 0xffffffffu);
    const float x = (float)(idx % (unsigned)W), y = (float)(idx / (unsigned)W);
    if (o < f.cap) {
      f.new_xy[2 * (bn + o)] = x;
      f.new_xy[2 * (bn + o) + 1] = y;
    }
    const int a0 = surv0 + o;
    if (a0 < f.cap) {
      f.list_xy[2 * (out0 + a0)] = x;
      f.list_xy[2 * (out0 + a0) + 1] = y;
      f.list_id[out0 + a0] = id0 + o;
    }
    if (!f.stereo_after && (r == 0 ? ss0 : (int)f.spec_status[q]) == VIO_TRACK_OK) {
      const int a1 = surv1 + om++;
      if (a1 < f.cap) {
        f.list_xy[2 * (out0 + cap + a1)] = r == 0 ? sx0 : f.spec_xy[2 * q];
        f.list_xy[2 * (out0 + cap + a1) + 1] = r == 0 ? sy0 : f.spec_xy[2 * q + 1];
        f.list_id[out0 + cap + a1] = id0 + o;
      }
    }
  }
  const int c0 = min(surv0 + new_tot, f.cap);
  const int c1 = min(surv1 + m_tot, f.cap);
  if (slot_ok) {
    f.list_status[out0 + t] = t < c0 ? VIO_TRACK_OK : VIO_TRACK_EMPTY;
    f.list_status[out0 + cap + t] = t < c1 ? VIO_TRACK_OK : VIO_TRACK_EMPTY;
  }
  if (t == 0) {
    f.list_count[cnt_out] = c0;
    f.list_count[cnt_out + 1] = c1;
    f.new_count[s] = min(new_tot, f.cap);
    f.next_id[s] = id0 + new_tot;
    st[VIO_STAT_TRK0] = n0;
    st[VIO_STAT_TRK1] = n1;
    st[VIO_STAT_OK0] = surv0;
    st[VIO_STAT_OK1] = surv1;
    st[VIO_STAT_NEW] = new_tot;
    st[VIO_STAT_MATCHED] = m_tot;
    st[VIO_STAT_CAND] = c_tot;
    st[VIO_STAT_LEARNED] = learned_s;
    if (f.slotted && !f.stereo_after) {   // else the append kernel ends the step
      f.parity[s] = sr.lo;
      f.have_prev[s] = 1;
    }
  }
}

// The finalisation of stream s of launch f (one CTA of K3_THREADS threads):
// survivors, occupancy, per-cell selection, appends, counts and statistics.
// occ_s: shared memory of one int per cell; ws32, ws64: K3_THREADS / 32
// entries each.
__device__ __forceinline__ void finalize_stream(const FrameLaunch& f, int s, int* occ_s,
                                                int* ws32, unsigned long long* ws64) {
  const StreamRef sr = stream_ref(f, s);
  const int k = f.p.k_per_cell;
  const int gx = f.g.w[0] / f.p.cell_w, gy = f.g.h[0] / f.p.cell_h;
  const int n_cells = gx * gy;
  const int W = f.g.w[0];
  const long long cap = f.cap;
  const int t = threadIdx.x;
  // this launch's step index + 1 (K1 incremented it)
  const int ctr = *(f.ctr_copy ? f.ctr_copy : f.step_ctr);
  int32_t* st = f.stats + ((long long)((ctr - 1) % VIO_STATS_RING) * f.n_streams + s) * VIO_N_STATS;
  if (!sr.active) {
    if (t < VIO_N_STATS) st[t] = 0;
    return;
  }
  if (f.cap <= K3_THREADS && n_cells <= K3_THREADS) {
    finalize_one_pass(f, s, sr, st, occ_s, reinterpret_cast<unsigned*>(ws32), ws64);
    return;
  }
  // the inputs of part 2 for this thread's first cell and its first
  // candidate, loaded now: they do not depend on part 1
  const long long cbase = (long long)s * n_cells;
  const int crun = (n_cells + K3_THREADS - 1) / K3_THREADS;
  const int pc = t * crun;
  const int id0 = f.next_id[s];
  int pre_nc = 0, pre_sst = 0;
  unsigned long long pre_key = 0;
  float pre_sx = 0.f, pre_sy = 0.f;
  if (pc < n_cells) {
    const long long q = (cbase + pc) * k;
    pre_nc = f.cand_count[cbase + pc];
    pre_key = f.cand[q];
    if (!f.stereo_after) {
      pre_sst = f.spec_status[q];
      pre_sx = f.spec_xy[2 * q];
      pre_sy = f.spec_xy[2 * q + 1];
    }
  }
  __shared__ int learned_s;
  for (int i = t; i < n_cells; i += K3_THREADS) occ_s[i] = 0;
  if (t == 0) learned_s = 0;
  __syncthreads();

  const long long in0 = (((long long)sr.li * f.n_streams + s) * 2) * cap;    // list in, camera 0
  const long long out0 = (((long long)sr.lo * f.n_streams + s) * 2) * cap;   // list out, camera 0
  const long long trk0 = (2LL * s) * cap;
  const long long cnt_in = ((long long)sr.li * f.n_streams + s) * 2;
  const long long cnt_out = ((long long)sr.lo * f.n_streams + s) * 2;

  // 1. survivors of temporal tracking of both cameras, in order: counts of
  //    the two cameras packed in one int (each < 2^15)
  const int n0 = sr.have_prev ? min(f.list_count[cnt_in], f.cap) : 0;
  const int n1 = sr.have_prev ? min(f.list_count[cnt_in + 1], f.cap) : 0;
  const int run = (max(n0, n1) + K3_THREADS - 1) / K3_THREADS;
  int surv0 = 0, surv1 = 0, n_learned = 0;
  for (int r0 = 0; r0 < run; r0 += kRunMax) {
    const int rl = min(kRunMax, run - r0);
    const int first = t * run + r0;
    unsigned keep0 = 0, keep1 = 0;
    // positions and ids of the first two entries, loaded with their status
    float ax0 = 0.f, ay0 = 0.f, ax1 = 0.f, ay1 = 0.f, bx0 = 0.f, by0 = 0.f, bx1 = 0.f, by1 = 0.f;
    int aid0 = 0, aid1 = 0, bid0 = 0, bid1 = 0;
    if (rl > 0) {
      const int i = first;
      if (i < n0) {
        ax0 = f.trk_xy[2 * (trk0 + i)];
        ay0 = f.trk_xy[2 * (trk0 + i) + 1];
        aid0 = f.list_id[in0 + i];
      }
      if (i < n1) {
        ax1 = f.trk_xy[2 * (trk0 + cap + i)];
        ay1 = f.trk_xy[2 * (trk0 + cap + i) + 1];
        aid1 = f.list_id[in0 + cap + i];
      }
    }
    if (rl > 1) {
      const int i = first + 1;
      if (i < n0) {
        bx0 = f.trk_xy[2 * (trk0 + i)];
        by0 = f.trk_xy[2 * (trk0 + i) + 1];
        bid0 = f.list_id[in0 + i];
      }
      if (i < n1) {
        bx1 = f.trk_xy[2 * (trk0 + cap + i)];
        by1 = f.trk_xy[2 * (trk0 + cap + i) + 1];
        bid1 = f.list_id[in0 + cap + i];
      }
    }
    for (int j = 0; j < rl; ++j) {
      const int i = first + j;
      if (i < n0 && f.trk_status[trk0 + i] == VIO_TRACK_OK) keep0 |= 1u << j;
      if (i < n1 && f.trk_status[trk0 + cap + i] == VIO_TRACK_OK) keep1 |= 1u << j;
      if (f.net) {
        if (keep0 & (1u << j)) n_learned += f.trk_learned[trk0 + i];
        if (keep1 & (1u << j)) n_learned += f.trk_learned[trk0 + cap + i];
      }
    }
    int tot;
    const int ex = block_scan<int>(__popc(keep0) | (__popc(keep1) << 16), ws32, tot);
    int o0 = surv0 + (ex & 0xffff), o1 = surv1 + (ex >> 16);
    for (int j = 0; j < rl; ++j) {
      const int i = first + j;
      if (keep0 & (1u << j)) {
        const float x = j == 0 ? ax0 : (j == 1 ? bx0 : f.trk_xy[2 * (trk0 + i)]);
        const float y = j == 0 ? ay0 : (j == 1 ? by0 : f.trk_xy[2 * (trk0 + i) + 1]);
        const long long d = out0 + o0++;
        f.list_xy[2 * d] = x;
        f.list_xy[2 * d + 1] = y;
        f.list_id[d] = j == 0 ? aid0 : (j == 1 ? bid0 : f.list_id[in0 + i]);
        if (x >= 0.f && y >= 0.f) {
          const int cx = cell_of(x, f.p.cell_w), cy = cell_of(y, f.p.cell_h);
          if (cx < gx && cy < gy) atomicAdd(&occ_s[cy * gx + cx], 1);
        }
      }
      if (keep1 & (1u << j)) {
        const long long d = out0 + cap + o1++;
        f.list_xy[2 * d] = j == 0 ? ax1 : (j == 1 ? bx1 : f.trk_xy[2 * (trk0 + cap + i)]);
        f.list_xy[2 * d + 1] =
            j == 0 ? ay1 : (j == 1 ? by1 : f.trk_xy[2 * (trk0 + cap + i) + 1]);
        f.list_id[d] = j == 0 ? aid1 : (j == 1 ? bid1 : f.list_id[in0 + cap + i]);
      }
    }
    surv0 += tot & 0xffff;
    surv1 += tot >> 16;
    __syncthreads();   // ws32 is reused by the next chunk
  }
  if (n_learned) atomicAdd(&learned_s, n_learned);
  __syncthreads();     // occupancy and learned_s complete

  // 2. per cell: selection (k_eff = k - occupancy), matched subset, and the
  //    candidates matched; three counts packed in 21-bit fields
  const long long bn = (long long)s * cap;
  int new_tot = 0, m_tot = 0, c_tot = 0;
  for (int r0 = 0; r0 < crun; r0 += kRunMax) {
    const int rl = min(kRunMax, crun - r0);
    const int first = t * crun + r0;
    unsigned long long packed = 0;
    for (int j = 0; j < rl; ++j) {
      const int cell = first + j;
      if (cell >= n_cells) break;
      const bool pre = r0 == 0 && j == 0;   // the prefetched cell
      const int nc = pre ? pre_nc : f.cand_count[cbase + cell];
      const int occ = min(occ_s[cell], 255);
      f.occupancy[cbase + cell] = (uint8_t)occ;
      const int nsel = max(0, min(k - occ, nc));
      int nm = 0;
      if (!f.stereo_after)
        for (int r = 0; r < nsel; ++r)
          nm += (pre && r == 0 ? pre_sst : (int)f.spec_status[(cbase + cell) * k + r]) ==
                VIO_TRACK_OK;
      packed += (unsigned long long)nsel | ((unsigned long long)nm << 21) |
                ((unsigned long long)nc << 42);
    }
    unsigned long long tot;
    const unsigned long long ex = block_scan<unsigned long long>(packed, ws64, tot);
    int o = new_tot + (int)(ex & 0x1fffff);
    int om = m_tot + (int)((ex >> 21) & 0x1fffff);
    for (int j = 0; j < rl; ++j) {
      const int cell = first + j;
      if (cell >= n_cells) break;
      const bool pre = r0 == 0 && j == 0;
      const int occ = min(occ_s[cell], 255);
      const int nsel = max(0, min(k - occ, pre ? pre_nc : (int)f.cand_count[cbase + cell]));
      for (int r = 0; r < nsel; ++r, ++o) {
        const long long q = (cbase + cell) * k + r;
        const bool pr = pre && r == 0;
        const unsigned idx = ~(unsigned)((pr ? pre_key : f.cand[q]) & 0xffffffffu);
        const float x = (float)(idx % (unsigned)W), y = (float)(idx / (unsigned)W);
        if (o < f.cap) {
          f.new_xy[2 * (bn + o)] = x;
          f.new_xy[2 * (bn + o) + 1] = y;
        }
        const int o0 = surv0 + o;
        if (o0 < f.cap) {
          f.list_xy[2 * (out0 + o0)] = x;
          f.list_xy[2 * (out0 + o0) + 1] = y;
          f.list_id[out0 + o0] = id0 + o;
        }
        if (!f.stereo_after && (pr ? pre_sst : (int)f.spec_status[q]) == VIO_TRACK_OK) {
          const int o1 = surv1 + om++;
          if (o1 < f.cap) {
            f.list_xy[2 * (out0 + cap + o1)] = pr ? pre_sx : f.spec_xy[2 * q];
            f.list_xy[2 * (out0 + cap + o1) + 1] = pr ? pre_sy : f.spec_xy[2 * q + 1];
            f.list_id[out0 + cap + o1] = id0 + o;
          }
        }
      }
    }
    new_tot += (int)(tot & 0x1fffff);
    m_tot += (int)((tot >> 21) & 0x1fffff);
    c_tot += (int)((tot >> 42) & 0x1fffff);
    __syncthreads();
  }
  const int c0 = min(surv0 + new_tot, f.cap);
  const int c1 = min(surv1 + m_tot, f.cap);
  for (int i = t; i < f.cap; i += K3_THREADS) {
    f.list_status[out0 + i] = i < c0 ? VIO_TRACK_OK : VIO_TRACK_EMPTY;
    f.list_status[out0 + cap + i] = i < c1 ? VIO_TRACK_OK : VIO_TRACK_EMPTY;
  }
  if (t == 0) {
    f.list_count[cnt_out] = c0;
    f.list_count[cnt_out + 1] = c1;
    f.new_count[s] = min(new_tot, f.cap);
    f.next_id[s] = id0 + new_tot;
    st[VIO_STAT_TRK0] = n0;
    st[VIO_STAT_TRK1] = n1;
    st[VIO_STAT_OK0] = surv0;
    st[VIO_STAT_OK1] = surv1;
    st[VIO_STAT_NEW] = new_tot;
    st[VIO_STAT_MATCHED] = m_tot;
    st[VIO_STAT_CAND] = c_tot;
    st[VIO_STAT_LEARNED] = learned_s;
    if (f.slotted && !f.stereo_after) {   // else the append kernel ends the step
      f.parity[s] = sr.lo;
      f.have_prev[s] = 1;
    }
  }
}

}  // namespace vio
