// Model-based start of a track (Sec. III-E): the warp starts where the
// camera model, the predicted pose and the keypoint's inverse depth put the
// sample pattern in the target image. One thread per keypoint: the keypoint
// and its 52 pattern points (a fronto-parallel patch at the keypoint's
// inverse depth) are back-projected through the source pinhole, moved by the
// relative pose and projected through the target pinhole; the start
// translation is the keypoint's projection and the start angle the
// least-squares rotation from the pattern offsets to the projected offsets.
#include "common.cuh"
#include "track_dev.cuh"

namespace vio {
namespace {

struct PredictArgs {
  vio_pinhole ks, kd;
  const vio_pose* pose;   // per image
  const float* pts;       // [img][cap] float2
  const float* rho;       // [img][cap]
  const int32_t* count;   // per image, or null
  int cap, n_images;
  float* init;            // [img][cap] float3
  uint8_t* valid;         // [img][cap], or null
};

// Projection of the source pixel (x, y) at depth z into the target; false if
// it is not in front of the target camera.
__device__ __forceinline__ bool project(const PredictArgs& a, const vio_pose& T, float x, float y,
                                        float z, float& u, float& v) {
  const float X = (x - a.ks.cx) * (z / a.ks.fx), Y = (y - a.ks.cy) * (z / a.ks.fy);
  const float qx = T.R[0] * X + T.R[1] * Y + T.R[2] * z + T.t[0];
  const float qy = T.R[3] * X + T.R[4] * Y + T.R[5] * z + T.t[1];
  const float qz = T.R[6] * X + T.R[7] * Y + T.R[8] * z + T.t[2];
  if (!(qz > 0.f)) return false;
  const float iz = 1.f / qz;
  u = a.kd.fx * qx * iz + a.kd.cx;
  v = a.kd.fy * qy * iz + a.kd.cy;
  return true;
}

__global__ void predict_kernel(const __grid_constant__ PredictArgs a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)a.n_images * a.cap) return;
  const int img = (int)(i / a.cap), k = (int)(i - (long long)img * a.cap);
  const int n = a.count ? min(max(a.count[img], 0), a.cap) : a.cap;
  if (k >= n) {
    if (a.valid) a.valid[i] = 0;
    return;
  }
  const vio_pose T = a.pose[img];
  const float px = a.pts[2 * i], py = a.pts[2 * i + 1];
  const float rho = a.rho[i];
  float tx = px, ty = py, th = 0.f;
  bool ok = rho > 0.f;
  if (ok) {
    const float z = 1.f / rho;
    ok = project(a, T, px, py, z, tx, ty);
    float dot = 0.f, cross = 0.f;
    constexpr trk::Pattern P = trk::make_pattern();
#pragma unroll
    for (int j = 0; j < trk::kNP; ++j) {
      const float u = P.u[j], v = P.v[j];
      float yx = tx, yy = ty;
      ok = project(a, T, px + u, py + v, z, yx, yy) && ok;
      const float dx = yx - tx, dy = yy - ty;
      dot += u * dx + v * dy;
      cross += u * dy - v * dx;
    }
    if (ok) th = atan2f(cross, dot);
  }
  if (!ok) {
    tx = px;
    ty = py;
    th = 0.f;
  }
  a.init[3 * i] = tx;
  a.init[3 * i + 1] = ty;
  a.init[3 * i + 2] = th;
  if (a.valid) a.valid[i] = ok ? 1 : 0;
}

bool pinhole_ok(const vio_pinhole* k) {
  return k && k->fx > 0.f && k->fy > 0.f && k->cx == k->cx && k->cy == k->cy;
}

}  // namespace
}  // namespace vio

extern "C" vio_status vio_predict_warp(const vio_pinhole* k_src, const vio_pinhole* k_dst,
                                       const vio_pose* d_pose, const float* d_pts,
                                       const float* d_inv_depth, const int32_t* d_count,
                                       int32_t capacity, int32_t n_images, float* d_init,
                                       uint8_t* d_valid, void* stream) {
  if (!vio::pinhole_ok(k_src) || !vio::pinhole_ok(k_dst) || !d_pose || !d_pts ||
      !d_inv_depth || !d_init || capacity < 0 || n_images < 0)
    return VIO_ERR_INVALID_ARG;
  const long long total = (long long)capacity * n_images;
  if (total == 0) return VIO_OK;
  vio::PredictArgs a{*k_src, *k_dst, d_pose, d_pts, d_inv_depth, d_count, capacity, n_images,
                     d_init, d_valid};
  const int threads = 128;
  const long long blocks = (total + threads - 1) / threads;
  if (blocks > 0x7fffffffLL) return VIO_ERR_UNSUPPORTED;
  vio::predict_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(a);
  return cudaGetLastError() == cudaSuccess ? VIO_OK : VIO_ERR_CUDA;
}
