// Serving loop over a vio_batch (host runtime; the paper has no serving
// layer). Sessions are client stereo streams of a few size classes; each
// class is one group of the batch with a fixed number of resident slots,
// sized from a device-memory budget. A session holds a slot from admission
// to close (its pyramids, lists and frame slots stay on the device), and
// waits in its class's FIFO while no slot is free.
//
// Continuous batching: frames are uploaded as they arrive (pinned host ->
// a per-slot staging buffer, on the upload stream, overlapping the steps in
// flight); while fewer than two steps are in flight, every admitted session
// with an uploaded frame joins the next step: staging -> its batch slot
// (device to device, on the compute stream after the upload's event), one
// batch step (its captured graph), then the lists of the groups in the step
// are read back into one of two sets of pinned buffers before the step's
// completion event. With two steps in flight the GPU goes from one step to
// the next without waiting for the host; a session can be in both (its
// frames run in stream order). Completions carry the frame's arrival, launch
// and completion times.
#include <pthread.h>
#include <sched.h>
#include <string.h>

#include <chrono>
#include <deque>
#include <new>
#include <vector>

#include "frame.cuh"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
  const uint8_t* host;
  double t_arrival;
  int64_t tag;
  int32_t flags;
};

struct Session {
  int cls = -1, slot = -1;
  bool open = false, closing = false;
  std::deque<Req> queue;               // arrived, not yet uploaded
  float* out_xy = nullptr;             // caller's host buffers (optional)
  int32_t* out_id = nullptr;
  int32_t* out_count = nullptr;
};

enum StageState { kFree = 0, kUploaded = 1, kInStep = 2 };

struct Slot {
  int64_t session = -1;
  uint8_t* staging[2] = {nullptr, nullptr};
  cudaEvent_t up_ev[2] = {nullptr, nullptr};
  int state[2] = {kFree, kFree};
  Req req[2];
  int order = 0;                       // staging buffer of the oldest uploaded frame
};

constexpr int kInFlight = 2;

struct Class {
  vio_stream_group spec;
  size_t frame_bytes = 0;
  std::vector<Slot> slots;
  std::deque<int64_t> waiting;
  // pinned copies of the group's outputs after a step (one set per step in flight)
  float* h_xy[kInFlight] = {};
  int32_t* h_id[kInFlight] = {};
  int32_t* h_count[kInFlight] = {};
  int32_t* h_new[kInFlight] = {};
};

struct Member {
  int cls, slot, buf;
  int64_t session;
  Req req;
};

struct StepRec {
  std::vector<Member> members;
  std::vector<std::vector<int32_t>> parity;   // per class, list parity after the step
  double t_launch = 0;
  int out = 0;                                // output buffer set and event index
};

}  // namespace

struct vio_server {
  vio_batch* batch = nullptr;
  std::vector<Class> cls;
  std::vector<Session> sessions;
  cudaStream_t cs = nullptr, us = nullptr;
  cudaEvent_t step_ev[kInFlight] = {};
  std::deque<StepRec> flight;
  int next_out = 0;
  std::vector<int32_t> active;
  std::vector<vio_server_done> done;
  std::vector<int64_t> closing;        // sessions closing while they hold a slot
  uint8_t* d_staging = nullptr;
  int64_t steps = 0;
  int64_t budget = 0, used = 0;
  double loop_max_gap = 0.0;           // host loop of the last trace
  int64_t loop_over_1ms = 0;
  int32_t pin_cpu = -1, rt_priority = 0;   // loop scheduling asked for
  int32_t granted = 0;                     // what the last trace got (bit 0 pin, bit 1 RT)
};

namespace {

int64_t slot_bytes(const vio_stream_group& g) {
  vio_stream_group one = g;
  one.n_streams = 1;
  int64_t b = 0;
  if (vio_batch_device_bytes(&one, 1, &b) != VIO_OK) return -1;
  return b + 2 * 2 * (int64_t)g.w * g.h + 512;   // plus two staging frames
}

int stream_index(const vio_server* s, int c, int j) {
  int k = 0;
  for (int i = 0; i < c; ++i) k += (int)s->cls[i].slots.size();
  return k + j;
}

void admit_waiting(vio_server* s, int c) {
  Class& C = s->cls[c];
  for (size_t j = 0; j < C.slots.size() && !C.waiting.empty(); ++j) {
    if (C.slots[j].session >= 0) continue;
    const int64_t id = C.waiting.front();
    C.waiting.pop_front();
    C.slots[j].session = id;
    s->sessions[id].slot = (int)j;
    if (s->sessions[id].closing) s->closing.push_back(id);
    vio_batch_reset_stream(s->batch, c, (int)j, s->cs);   // a new stream starts fresh
  }
}

void release_if_done(vio_server* s, int64_t id) {
  Session& S = s->sessions[id];
  if (!S.closing || S.slot < 0 || !S.queue.empty()) return;
  Slot& L = s->cls[S.cls].slots[S.slot];
  if (L.state[0] != kFree || L.state[1] != kFree) return;
  L.session = -1;
  S.slot = -1;
  S.open = false;
  admit_waiting(s, S.cls);
}

// Releases the slots of closing sessions whose frames are all done.
void release_closing(vio_server* s) {
  std::vector<int64_t> cur;
  cur.swap(s->closing);           // admissions below append to s->closing
  for (int64_t id : cur) {
    release_if_done(s, id);
    if (s->sessions[id].slot >= 0) s->closing.push_back(id);
  }
}

// Completion of the oldest step in flight: records, caller outputs, stage
// buffers.
void complete_step(vio_server* s, int32_t status) {
  const double t = now_s();
  const StepRec& R = s->flight.front();
  for (const Member& m : R.members) {
    Class& C = s->cls[m.cls];
    Slot& L = C.slots[m.slot];
    Session& S = s->sessions[m.session];
    vio_server_done d{};
    d.session = m.session;
    d.tag = m.req.tag;
    d.t_arrival = m.req.t_arrival;
    d.t_launch = R.t_launch;
    d.t_done = t;
    d.status = status;
    if (status == VIO_OK) {
      const int ns = C.spec.n_streams, cap = C.spec.capacity, o = R.out;
      const int q = R.parity[m.cls][m.slot];
      const size_t base = ((size_t)q * ns + m.slot) * 2;
      d.n_tracks[0] = C.h_count[o][base];
      d.n_tracks[1] = C.h_count[o][base + 1];
      d.n_new = C.h_new[o][m.slot];
      if (S.out_count) {
        S.out_count[0] = d.n_tracks[0];
        S.out_count[1] = d.n_tracks[1];
      }
      for (int c = 0; c < 2; ++c) {
        const size_t off = (base + c) * cap;
        const int n = d.n_tracks[c] < cap ? d.n_tracks[c] : cap;
        if (S.out_xy)
          memcpy(S.out_xy + 2 * (size_t)c * cap, C.h_xy[o] + 2 * off, (size_t)n * 8);
        if (S.out_id) memcpy(S.out_id + (size_t)c * cap, C.h_id[o] + off, (size_t)n * 4);
      }
    }
    s->done.push_back(d);
    L.state[m.buf] = kFree;
  }
  s->flight.pop_front();
  release_closing(s);
}

// Completion of every step in flight whose event has passed (in order).
vio_status drain(vio_server* s, bool wait) {
  while (!s->flight.empty()) {
    cudaEvent_t ev = s->step_ev[s->flight.front().out];
    const cudaError_t e = wait ? cudaEventSynchronize(ev) : cudaEventQuery(ev);
    if (e == cudaErrorNotReady) return VIO_OK;
    if (e != cudaSuccess) {
      cudaGetLastError();
      while (!s->flight.empty()) complete_step(s, VIO_ERR_CUDA);
      return VIO_ERR_CUDA;
    }
    complete_step(s, VIO_OK);
  }
  return VIO_OK;
}

// Uploads of arrived frames into free staging buffers.
vio_status start_uploads(vio_server* s) {
  for (size_t c = 0; c < s->cls.size(); ++c) {
    Class& C = s->cls[c];
    for (Slot& L : C.slots) {
      if (L.session < 0) continue;
      Session& S = s->sessions[L.session];
      // buffers fill from L.order on, so the oldest uploaded frame is always
      // the one at L.order (a launch takes it and moves L.order on)
      for (int k = 0; k < 2 && !S.queue.empty(); ++k) {
        const int b = (L.order + k) & 1;
        if (L.state[b] != kFree) continue;
        const Req r = S.queue.front();
        if (cudaMemcpyAsync(L.staging[b], r.host, C.frame_bytes, cudaMemcpyHostToDevice,
                            s->us) != cudaSuccess ||
            cudaEventRecord(L.up_ev[b], s->us) != cudaSuccess)
          return VIO_ERR_CUDA;
        L.state[b] = kUploaded;
        L.req[b] = r;
        S.queue.pop_front();
      }
    }
  }
  return VIO_OK;
}

vio_status launch_step(vio_server* s) {
  StepRec R;
  std::fill(s->active.begin(), s->active.end(), 0);
  for (size_t c = 0; c < s->cls.size(); ++c) {
    Class& C = s->cls[c];
    for (size_t j = 0; j < C.slots.size(); ++j) {
      Slot& L = C.slots[j];
      if (L.session < 0) continue;
      const int b = L.order;
      if (L.state[b] != kUploaded) continue;
      uint8_t* d_frame = nullptr;
      if (vio_batch_next_frame(s->batch, (int)c, (int)j, &d_frame) != VIO_OK ||
          cudaStreamWaitEvent(s->cs, L.up_ev[b], 0) != cudaSuccess ||
          cudaMemcpyAsync(d_frame, L.staging[b], C.frame_bytes, cudaMemcpyDeviceToDevice,
                          s->cs) != cudaSuccess)
        return VIO_ERR_CUDA;
      L.state[b] = kInStep;
      L.order ^= 1;
      R.members.push_back(Member{(int)c, (int)j, b, L.session, L.req[b]});
      s->active[stream_index(s, (int)c, (int)j)] = 1;
    }
  }
  if (R.members.empty()) return VIO_OK;
  R.t_launch = now_s();
  R.out = s->next_out;
  R.parity.resize(s->cls.size());
  s->flight.push_back(R);          // from here on a failure completes it with the error
  StepRec& F = s->flight.back();
  vio_status st = vio_batch_step(s->batch, s->active.data(), s->cs);
  if (st != VIO_OK) return st;
  std::vector<char> has(s->cls.size(), 0);
  for (const Member& m : F.members) has[m.cls] = 1;
  const int o = F.out;
  for (size_t c = 0; c < s->cls.size(); ++c) {
    if (!has[c]) continue;
    Class& C = s->cls[c];
    vio_frontend_view v;
    F.parity[c].assign(C.slots.size(), 0);
    if (vio_batch_get_view(s->batch, (int)c, &v, F.parity[c].data()) != VIO_OK)
      return VIO_ERR_CUDA;
    const size_t ns = C.spec.n_streams, cap = C.spec.capacity, lists = 2 * ns * 2;
    if (cudaMemcpyAsync(C.h_count[o], v.d_track_count, lists * 4, cudaMemcpyDeviceToHost,
                        s->cs) != cudaSuccess ||
        cudaMemcpyAsync(C.h_new[o], v.d_new_count, ns * 4, cudaMemcpyDeviceToHost, s->cs) !=
            cudaSuccess ||
        cudaMemcpyAsync(C.h_xy[o], v.d_track_xy, lists * cap * 8, cudaMemcpyDeviceToHost,
                        s->cs) != cudaSuccess ||
        cudaMemcpyAsync(C.h_id[o], v.d_track_id, lists * cap * 4, cudaMemcpyDeviceToHost,
                        s->cs) != cudaSuccess)
      return VIO_ERR_CUDA;
  }
  if (cudaEventRecord(s->step_ev[o], s->cs) != cudaSuccess) return VIO_ERR_CUDA;
  s->next_out ^= 1;
  ++s->steps;
  return VIO_OK;
}

void destroy(vio_server* s) {
  if (!s) return;
  if (s->cs) cudaStreamSynchronize(s->cs);
  if (s->us) cudaStreamSynchronize(s->us);
  for (Class& C : s->cls) {
    for (Slot& L : C.slots)
      for (int b = 0; b < 2; ++b)
        if (L.up_ev[b]) cudaEventDestroy(L.up_ev[b]);
    for (int o = 0; o < kInFlight; ++o) {
      cudaFreeHost(C.h_xy[o]);
      cudaFreeHost(C.h_id[o]);
      cudaFreeHost(C.h_count[o]);
      cudaFreeHost(C.h_new[o]);
    }
  }
  if (s->batch) vio_batch_destroy(s->batch);
  cudaFree(s->d_staging);
  for (int o = 0; o < kInFlight; ++o)
    if (s->step_ev[o]) cudaEventDestroy(s->step_ev[o]);
  if (s->cs) cudaStreamDestroy(s->cs);
  if (s->us) cudaStreamDestroy(s->us);
  delete s;
}

}  // namespace

extern "C" double vio_server_now(void) { return now_s(); }

extern "C" vio_status vio_server_plan(const vio_stream_group* classes, int32_t n_classes,
                                      int64_t budget_bytes, int32_t* slots_out,
                                      int64_t* bytes_out) {
  if (!classes || !slots_out || n_classes < 1 || n_classes > vio::kMaxGroups || budget_bytes < 0)
    return VIO_ERR_INVALID_ARG;
  std::vector<int64_t> per(n_classes);
  int64_t want = 0;
  for (int k = 0; k < n_classes; ++k) {
    if (classes[k].n_streams < 1) return VIO_ERR_INVALID_ARG;
    per[k] = slot_bytes(classes[k]);
    if (per[k] < 0) return VIO_ERR_INVALID_ARG;
    want += per[k] * classes[k].n_streams;
  }
  // every class keeps at least one slot; beyond that the slots scale down
  // together until the budget holds them
  int64_t total = 0;
  for (int k = 0; k < n_classes; ++k) {
    int64_t n = classes[k].n_streams;
    if (want > budget_bytes) n = (int64_t)((double)n * (double)budget_bytes / (double)want);
    if (n < 1) n = 1;
    slots_out[k] = (int32_t)n;
    total += n * per[k];
  }
  if (bytes_out) *bytes_out = total;
  return total <= budget_bytes ? VIO_OK : VIO_ERR_OOM;
}

extern "C" vio_status vio_server_create(vio_server** out, const vio_stream_group* classes,
                                        int32_t n_classes, int64_t budget_bytes) {
  if (!out) return VIO_ERR_INVALID_ARG;
  *out = nullptr;
  std::vector<int32_t> slots(n_classes > 0 ? n_classes : 1);
  int64_t bytes = 0;
  vio_status st = vio_server_plan(classes, n_classes, budget_bytes, slots.data(), &bytes);
  if (st != VIO_OK) return st;
  vio_server* s = new (std::nothrow) vio_server();
  if (!s) return VIO_ERR_OOM;
  s->budget = budget_bytes;
  s->used = bytes;
  std::vector<vio_stream_group> groups(classes, classes + n_classes);
  size_t staging = 0;
  for (int k = 0; k < n_classes; ++k) {
    groups[k].n_streams = slots[k];
    staging += (size_t)slots[k] * 2 * 2 * groups[k].w * groups[k].h;
  }
  if (vio_batch_create(&s->batch, groups.data(), n_classes) != VIO_OK ||
      cudaMalloc(&s->d_staging, staging) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->us, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->step_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->step_ev[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    destroy(s);
    return VIO_ERR_OOM;
  }
  vio_batch_set_graph(s->batch, 1);
  {
    // steps hold a frame or two: score each detection cell with 4 warps
    vio_batch_tune t;
    vio_batch_get_tune(s->batch, &t);
    t.det_warps = 4;
    vio_batch_set_tune(s->batch, &t);
  }
  uint8_t* q = s->d_staging;
  int total = 0;
  s->cls.resize(n_classes);
  for (int k = 0; k < n_classes; ++k) {
    Class& C = s->cls[k];
    C.spec = groups[k];
    C.frame_bytes = (size_t)2 * C.spec.w * C.spec.h;
    C.slots.resize(slots[k]);
    for (Slot& L : C.slots)
      for (int b = 0; b < 2; ++b) {
        L.staging[b] = q;
        q += C.frame_bytes;
        if (cudaEventCreateWithFlags(&L.up_ev[b], cudaEventDisableTiming) != cudaSuccess) {
          destroy(s);
          return VIO_ERR_CUDA;
        }
      }
    const size_t lists = (size_t)2 * slots[k] * 2, cap = C.spec.capacity;
    for (int o = 0; o < kInFlight; ++o)
      if (cudaMallocHost(&C.h_xy[o], lists * cap * 8) != cudaSuccess ||
          cudaMallocHost(&C.h_id[o], lists * cap * 4) != cudaSuccess ||
          cudaMallocHost(&C.h_count[o], lists * 4) != cudaSuccess ||
          cudaMallocHost(&C.h_new[o], (size_t)slots[k] * 4) != cudaSuccess) {
        cudaGetLastError();
        destroy(s);
        return VIO_ERR_OOM;
      }
    total += slots[k];
  }
  s->active.assign(total, 0);
  *out = s;
  return VIO_OK;
}

extern "C" vio_status vio_server_destroy(vio_server* s) {
  if (!s) return VIO_ERR_INVALID_ARG;
  destroy(s);
  return VIO_OK;
}

extern "C" vio_status vio_server_slots(const vio_server* s, int32_t cls, int32_t* n_slots,
                                       int64_t* device_bytes) {
  if (!s || cls < 0 || cls >= (int)s->cls.size()) return VIO_ERR_INVALID_ARG;
  if (n_slots) *n_slots = (int32_t)s->cls[cls].slots.size();
  if (device_bytes) *device_bytes = s->used;
  return VIO_OK;
}

extern "C" vio_status vio_server_set_initnet(vio_server* s, const void* d_packed,
                                             const vio_initnet_cfg* cfg) {
  if (!s) return VIO_ERR_INVALID_ARG;
  if (drain(s, true) != VIO_OK) return VIO_ERR_CUDA;
  return vio_batch_set_initnet(s->batch, d_packed, cfg);
}

extern "C" vio_status vio_server_set_tune(vio_server* s, const vio_batch_tune* t) {
  if (!s) return VIO_ERR_INVALID_ARG;
  if (drain(s, true) != VIO_OK) return VIO_ERR_CUDA;
  return vio_batch_set_tune(s->batch, t);
}

extern "C" vio_status vio_server_open(vio_server* s, int32_t cls, int64_t* session,
                                      int32_t* admitted) {
  if (!s || !session || cls < 0 || cls >= (int)s->cls.size()) return VIO_ERR_INVALID_ARG;
  const int64_t id = (int64_t)s->sessions.size();
  s->sessions.emplace_back();
  Session& S = s->sessions.back();
  S.cls = cls;
  S.open = true;
  s->cls[cls].waiting.push_back(id);
  admit_waiting(s, cls);
  *session = id;
  if (admitted) *admitted = s->sessions[id].slot >= 0;
  return VIO_OK;
}

extern "C" vio_status vio_server_set_output(vio_server* s, int64_t session, float* host_xy,
                                            int32_t* host_id, int32_t* host_count) {
  if (!s || session < 0 || session >= (int64_t)s->sessions.size()) return VIO_ERR_INVALID_ARG;
  Session& S = s->sessions[session];
  S.out_xy = host_xy;
  S.out_id = host_id;
  S.out_count = host_count;
  return VIO_OK;
}

extern "C" vio_status vio_server_submit(vio_server* s, int64_t session,
                                        const uint8_t* host_frame, double t_arrival, int64_t tag,
                                        int32_t flags) {
  if (!s || !host_frame || session < 0 || session >= (int64_t)s->sessions.size())
    return VIO_ERR_INVALID_ARG;
  Session& S = s->sessions[session];
  if (!S.open || S.closing) return VIO_ERR_INVALID_ARG;
  S.queue.push_back(Req{host_frame, t_arrival, tag, flags});
  if (flags & VIO_SERVER_LAST) {
    S.closing = true;
    if (S.slot >= 0) s->closing.push_back(session);
  }
  return VIO_OK;
}

extern "C" vio_status vio_server_close(vio_server* s, int64_t session) {
  if (!s || session < 0 || session >= (int64_t)s->sessions.size()) return VIO_ERR_INVALID_ARG;
  Session& S = s->sessions[session];
  if (!S.open) return VIO_OK;
  S.closing = true;
  if (S.slot < 0) {               // still waiting: leave the queue
    auto& w = s->cls[S.cls].waiting;
    for (auto it = w.begin(); it != w.end(); ++it)
      if (*it == session) {
        w.erase(it);
        break;
      }
    S.queue.clear();
    S.open = false;
    return VIO_OK;
  }
  s->closing.push_back(session);
  release_closing(s);
  return VIO_OK;
}

extern "C" vio_status vio_server_poll(vio_server* s, int32_t* n_done) {
  if (!s) return VIO_ERR_INVALID_ARG;
  vio_status st = drain(s, false);
  if (st == VIO_OK) st = start_uploads(s);
  if (st == VIO_OK && (int)s->flight.size() < kInFlight) {
    st = launch_step(s);
    if (st != VIO_OK) {   // report the frames of the failed step and of any before it
      cudaStreamSynchronize(s->cs);
      cudaGetLastError();
      while (!s->flight.empty()) complete_step(s, st);
    }
  }
  if (n_done) *n_done = (int32_t)s->done.size();
  return st;
}

extern "C" int32_t vio_server_take(vio_server* s, vio_server_done* out, int32_t max) {
  if (!s || !out || max <= 0) return 0;
  const int32_t n = (int32_t)std::min<size_t>((size_t)max, s->done.size());
  for (int32_t i = 0; i < n; ++i) out[i] = s->done[i];
  s->done.erase(s->done.begin(), s->done.begin() + n);
  return n;
}

extern "C" vio_status vio_server_loop_stats(const vio_server* s, double* max_gap_s,
                                           int64_t* n_over_1ms) {
  if (!s || !max_gap_s || !n_over_1ms) return VIO_ERR_INVALID_ARG;
  *max_gap_s = s->loop_max_gap;
  *n_over_1ms = s->loop_over_1ms;
  return VIO_OK;
}

extern "C" vio_status vio_server_run_trace(vio_server* s, const vio_server_req* reqs,
                                           int64_t n, vio_server_done* out, double timeout_s,
                                           int64_t* n_steps) {
  if (!s || (!reqs && n) || (!out && n) || n < 0) return VIO_ERR_INVALID_ARG;
  for (int64_t i = 1; i < n; ++i)
    if (reqs[i].t_offset < reqs[i - 1].t_offset) return VIO_ERR_INVALID_ARG;
  const int64_t steps0 = s->steps;
  // the loop's thread: pinned to one CPU and at a real-time priority for the
  // call where asked and permitted (restored on return)
  s->granted = 0;
  const pthread_t self = pthread_self();
  cpu_set_t old_set;
  bool pinned = false;
  if (s->pin_cpu != -1 && pthread_getaffinity_np(self, sizeof(old_set), &old_set) == 0) {
    const int cpu = s->pin_cpu == -2 ? sched_getcpu() : s->pin_cpu;
    if (cpu >= 0 && cpu < CPU_SETSIZE) {
      cpu_set_t one;
      CPU_ZERO(&one);
      CPU_SET(cpu, &one);
      pinned = pthread_setaffinity_np(self, sizeof(one), &one) == 0;
    }
  }
  int old_policy = 0;
  sched_param old_param{};
  bool rt = false;
  if (s->rt_priority > 0 && pthread_getschedparam(self, &old_policy, &old_param) == 0) {
    sched_param p{};
    p.sched_priority = s->rt_priority;
    rt = pthread_setschedparam(self, SCHED_FIFO, &p) == 0;
  }
  s->granted = (pinned ? 1 : 0) | (rt ? 2 : 0);
  const double t0 = now_s();
  int64_t next = 0, got = 0;
  vio_status st = VIO_OK;
  s->loop_max_gap = 0.0;
  s->loop_over_1ms = 0;
  double t_prev = 0.0;
  while (got < n) {
    const double t = now_s() - t0;
    const double gap = t - t_prev;
    t_prev = t;
    if (gap > s->loop_max_gap) s->loop_max_gap = gap;
    if (gap > 1e-3) ++s->loop_over_1ms;
    if (t > timeout_s) {
      st = VIO_ERR_TIMEOUT;
      break;
    }
    while (next < n && reqs[next].t_offset <= t) {
      const vio_server_req& r = reqs[next];
      st = vio_server_submit(s, r.session, r.host_frame, t0 + r.t_offset, r.tag, r.flags);
      if (st != VIO_OK) break;
      ++next;
    }
    if (st != VIO_OK) break;
    int32_t nd = 0;
    const vio_status ps = vio_server_poll(s, &nd);
    if (ps != VIO_OK && st == VIO_OK) st = ps;
    got += vio_server_take(s, out + got, (int32_t)(n - got));
    if (st != VIO_OK) break;
  }
  if (rt) pthread_setschedparam(self, old_policy, &old_param);
  if (pinned) pthread_setaffinity_np(self, sizeof(old_set), &old_set);
  if (n_steps) *n_steps = s->steps - steps0;
  return st;
}

extern "C" vio_status vio_server_set_loop_policy(vio_server* s, int32_t pin_cpu,
                                                 int32_t rt_priority) {
  if (!s || pin_cpu < -2 || rt_priority < 0 || rt_priority > 99) return VIO_ERR_INVALID_ARG;
  s->pin_cpu = pin_cpu;
  s->rt_priority = rt_priority;
  return VIO_OK;
}

extern "C" vio_status vio_server_loop_policy_granted(const vio_server* s, int32_t* granted) {
  if (!s || !granted) return VIO_ERR_INVALID_ARG;
  *granted = s->granted;
  return VIO_OK;
}
