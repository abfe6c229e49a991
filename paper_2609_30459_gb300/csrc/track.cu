// Pyramidal inverse-compositional KLT (Sec. III-E, Eq. 4-5) for the stage
// entry points vio_track_patches / vio_stereo_match, and the
// forward-backward distance check. The tracker itself is in track_dev.cuh.
#include "track_dev.cuh"

namespace vio {
namespace {

struct TrackArgs {
  Geom g;
  Batch src, dst;
  const float* pts;    // float2 per slot
  const float* init;   // float3 per slot or null
  const int32_t* count;
  int capacity, n_images;
  TrackCfg cfg;
  float* out3;         // float3 per slot or null
  float* out2;         // float2 per slot or null
  uint8_t* status;
  float* fb_dist;
  float* last_step;    // per slot or null
  int shared_pts;      // 1: every image tracks the same keypoints (pts, count of image 0)
};

constexpr int TRK_THREADS = 128;

__global__ void __launch_bounds__(TRK_THREADS) track_kernel(TrackArgs a) {
  const long long wid = ((long long)blockIdx.x * TRK_THREADS + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long total = (long long)a.capacity * a.n_images;
  if (wid >= total) return;
  const int img = (int)(wid / a.capacity);
  const int k = (int)(wid - (long long)img * a.capacity);
  const int n = a.count ? min(a.count[a.shared_pts ? 0 : img], a.capacity) : a.capacity;
  const long long pk = a.shared_pts ? k : wid;   // keypoint slot of the source list
  const float nanf_ = __int_as_float(0x7fc00000);
  if (k >= n) {
    if (lane == 0) {
      a.status[wid] = VIO_TRACK_EMPTY;
      if (a.out3) a.out3[3 * wid] = a.out3[3 * wid + 1] = a.out3[3 * wid + 2] = nanf_;
      if (a.out2) a.out2[2 * wid] = a.out2[2 * wid + 1] = nanf_;
      if (a.fb_dist) a.fb_dist[wid] = nanf_;
      if (a.last_step) a.last_step[wid] = nanf_;
    }
    return;
  }
  trk::Pos tf;
  float thf = 0.f, dist, last = 0.f;
  bool have;
  const bool hi = a.init != nullptr;
  const int st = trk::track_fb(a.g, a.src, img, a.dst, img, a.pts[2 * pk], a.pts[2 * pk + 1],
                               hi, hi ? a.init[3 * wid] : 0.f, hi ? a.init[3 * wid + 1] : 0.f,
                               hi ? a.init[3 * wid + 2] : 0.f, a.cfg, top_level(a.cfg, a.g),
                               lane, tf, thf, have, dist, last);
  if (lane == 0) {
    a.status[wid] = (uint8_t)st;
    const float ox = have ? (float)tf.ax + tf.dx : nanf_;
    const float oy = have ? (float)tf.ay + tf.dy : nanf_;
    if (a.out3) {
      a.out3[3 * wid] = ox;
      a.out3[3 * wid + 1] = oy;
      a.out3[3 * wid + 2] = have ? thf : nanf_;
    }
    if (a.out2) {
      a.out2[2 * wid] = ox;
      a.out2[2 * wid + 1] = oy;
    }
    if (a.fb_dist) a.fb_dist[wid] = dist;
    if (a.last_step) a.last_step[wid] = have ? last : nanf_;
  }
}

__global__ void fb_check_kernel(const float* __restrict__ orig, const float* __restrict__ back,
                                const int32_t* __restrict__ count, int capacity,
                                long long total, float max_dist, uint8_t* __restrict__ status,
                                float* __restrict__ dist) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int img = (int)(i / capacity);
  const int k = (int)(i - (long long)img * capacity);
  const int n = count ? min(count[img], capacity) : capacity;
  if (k >= n || status[i] != VIO_TRACK_OK) return;
  const float ex = back[3 * i] - orig[2 * i];
  const float ey = back[3 * i + 1] - orig[2 * i + 1];
  const float d = sqrtf(ex * ex + ey * ey);
  if (dist) dist[i] = d;
  if (!(d <= max_dist)) status[i] = VIO_TRACK_FB_FAIL;
}

}  // namespace

cudaError_t launch_track(const Geom& g, const Batch& src, const Batch& dst, const float* pts,
                         const float* init, const int32_t* count, int capacity,
                         const TrackCfg& cfg, float* out3, float* out2, uint8_t* status,
                         float* fb_dist, cudaStream_t s, bool shared_pts, float* last_step) {
  TrackArgs a{g,    src,  dst,    pts,     init,      count,
              capacity, src.n, cfg, out3, out2, status, fb_dist, last_step,
              shared_pts ? 1 : 0};
  const long long warps = (long long)capacity * src.n;
  if (warps == 0) return cudaSuccess;
  const long long blocks = (warps * 32 + TRK_THREADS - 1) / TRK_THREADS;
  track_kernel<<<(unsigned)blocks, TRK_THREADS, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fb_check(const float* orig, const float* back, const int32_t* count,
                            int capacity, int n_images, float max_dist, uint8_t* status,
                            float* dist, cudaStream_t s) {
  const long long total = (long long)capacity * n_images;
  if (total == 0) return cudaSuccess;
  fb_check_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(orig, back, count, capacity,
                                                                  total, max_dist, status, dist);
  return cudaGetLastError();
}

}  // namespace vio
