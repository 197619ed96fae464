// The terms of the layer-wise vectorisation loop (§4.2, adapted from LIVE):
//
//   k_udf_sums / k_udf_grad / k_udf_finish
//                    distance-weighted image loss: per pixel of a scene that
//                    received a new filled path, the distance d to that path's
//                    closed boundary polyline (the points nurbs_sample left in
//                    the workspace) gives the weight w = max(0, tau - d).  The
//                    scene's loss is sum w sum_c (I - I*)^2 / (C sum w); other
//                    scenes take the plain mean square error; the batch loss is
//                    the mean over scenes.  Pixels farther than tau from the
//                    path's padded box (which holds the polyline) have w = 0
//                    without a distance search.
//   k_xing           self-crossing penalty: one warp per curve sums
//                    max(0, -sigma sin_i) over the turns of the key-point
//                    polygon, sigma the sign of the polygon's total turn, and
//                    adds the gradient to the key points' x, y.
//   k_seed_rows / k_seed_windows
//                    per scene, the (2r+1)^2 window sums of the squared error
//                    (a row pass, then a column pass) and the pixel with the
//                    largest sum, first in row-major order on ties (a packed
//                    64-bit atomicMax: value bits above, inverted index below).
#include <cuda_runtime.h>

#include <algorithm>

#include "ns_internal.cuh"

namespace ns {

constexpr int kLiveThreads = 256;

// Distance from q to the closed polyline b[0..B) (segments b_k -> b_{k+1 mod B}).
__device__ __forceinline__ float polyline_distance(float qx, float qy, const float2* __restrict__ b, int B) {
  float best = 3.0e38f;
  float2 p0 = b[B - 1];
  for (int k = 0; k < B; ++k) {
    const float2 p1 = b[k];
    const float ex = p1.x - p0.x, ey = p1.y - p0.y;
    const float rx = qx - p0.x, ry = qy - p0.y;
    const float ee = ex * ex + ey * ey;
    const float t = ee > 0.f ? fminf(fmaxf((rx * ex + ry * ey) / ee, 0.f), 1.f) : 0.f;
    const float dx = rx - t * ex, dy = ry - t * ey;
    best = fminf(best, dx * dx + dy * dy);
    p0 = p1;
  }
  return sqrtf(best);
}

// Weight of one pixel centre for scene s (0 when the scene names no path).
__device__ __forceinline__ float udf_weight(const CurvePlan* __restrict__ plan, const float2* __restrict__ bpts,
                                            int nc, int c, float h, float tau, float qx, float qy) {
  if (c < 0 || c >= nc) return 0.f;
  const CurvePlan pl = plan[c];
  if (pl.kind != kFill || pl.M < 1) return 0.f;
  // the padded grid box holds the polyline: beyond tau of it the weight is 0
  const float bx0 = pl.x0, by0 = pl.y0, bx1 = pl.x0 + pl.nx * h, by1 = pl.y0 + pl.ny * h;
  const float ox = fmaxf(fmaxf(bx0 - qx, qx - bx1), 0.f), oy = fmaxf(fmaxf(by0 - qy, qy - by1), 0.f);
  if (ox * ox + oy * oy >= tau * tau) return 0.f;
  const float d = polyline_distance(qx, qy, bpts + pl.b_off, pl.M);
  return fmaxf(tau - d, 0.f);
}

struct UdfParams {
  int S, H, W, C, nc;
  float tau, h;
};

// Per-scene sums {sum w, sum w e, sum e}, e = sum_c (I - I*)^2.
__global__ void __launch_bounds__(kLiveThreads) k_udf_sums(UdfParams up, const CurvePlan* __restrict__ plan,
                                                           const float2* __restrict__ bpts,
                                                           const int* __restrict__ new_curve,
                                                           const float* __restrict__ image,
                                                           const float* __restrict__ target, float* sums) {
  grid_dep_wait();
  const long long hw = (long long)up.H * up.W;
  const long long n = hw * up.S;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long iters = (n + stride - 1) / stride;   // the same for every thread
  const int lane = threadIdx.x & 31;
  for (long long it = 0; it < iters; ++it) {
    const long long pix = it * stride + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool valid = pix < n;
    int s = -1;
    float e = 0.f;
    if (valid) {
      s = int(pix / hw);
      const int rem = int(pix - s * hw);
      const int y = rem / up.W, x = rem - y * up.W;
      for (int ch = 0; ch < up.C; ++ch) {
        const float d = image[pix * up.C + ch] - target[pix * up.C + ch];
        e = fmaf(d, d, e);
      }
      const float w = udf_weight(plan, bpts, up.nc, new_curve[s], up.h, up.tau, x + 0.5f, y + 0.5f);
      if (w > 0.f) {
        atomicAdd(sums + 4 * s + 0, w);
        atomicAdd(sums + 4 * s + 1, w * e);
      }
    }
    // the plain sum of squares: one atomic per warp when the warp is in one
    // scene (lane 0 holds the lowest pixel, so it is valid whenever any lane is)
    const int s0 = __shfl_sync(0xffffffffu, s, 0);
    if (__all_sync(0xffffffffu, !valid || s == s0)) {
      float v = e;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && s0 >= 0) atomicAdd(sums + 4 * s0 + 2, v);
    } else if (valid) {
      atomicAdd(sums + 4 * s + 2, e);
    }
  }
}

// The loss and, per scene, the gradient scale in the record's fourth slot:
// dL/dI = 2 scale w (I - I*) for a weighted scene, 2 |scale| (I - I*) for a
// plain one (stored negative to tell them apart).
__global__ void k_udf_finish(UdfParams up, const int* __restrict__ new_curve, float* sums, float* loss) {
  grid_dep_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float tot = 0.f;
  for (int s = 0; s < up.S; ++s) {
    float* sm = sums + 4 * s;
    const bool weighted = new_curve[s] >= 0 && new_curve[s] < up.nc && sm[0] > 0.f;
    if (weighted) {
      tot += sm[1] / (up.C * sm[0]);
      sm[3] = 1.f / (up.C * sm[0] * up.S);
    } else {
      tot += sm[2] / (float(up.C) * up.H * up.W);
      sm[3] = -1.f / (float(up.C) * up.H * up.W * up.S);
    }
  }
  *loss = tot / up.S;
}

__global__ void __launch_bounds__(kLiveThreads) k_udf_grad(UdfParams up, const CurvePlan* __restrict__ plan,
                                                           const float2* __restrict__ bpts,
                                                           const int* __restrict__ new_curve,
                                                           const float* __restrict__ image,
                                                           const float* __restrict__ target,
                                                           const float* __restrict__ sums, float* dimage) {
  grid_dep_wait();
  const long long hw = (long long)up.H * up.W;
  const long long n = hw * up.S;
  for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < n;
       pix += (long long)gridDim.x * blockDim.x) {
    const int s = int(pix / hw);
    const int rem = int(pix - s * hw);
    const int y = rem / up.W, x = rem - y * up.W;
    const float sc = sums[4 * s + 3];
    const float f = sc < 0.f ? -sc
                             : sc * udf_weight(plan, bpts, up.nc, new_curve[s], up.h, up.tau, x + 0.5f, y + 0.5f);
    for (int ch = 0; ch < up.C; ++ch) {
      const long long i = pix * up.C + ch;
      dimage[i] = 2.f * f * (image[i] - target[i]);
    }
  }
}

// One warp per curve: the self-crossing penalty of its key-point polygon.
__global__ void __launch_bounds__(128) k_xing(ns_curves cv, float lambda, float* loss, float* dkey) {
  grid_dep_wait();
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= cv.n_curves) return;
  const int k0 = cv.key_offset[c];
  const int nk = cv.key_offset[c + 1] - k0;
  const bool closed = (cv.flags[c] & NS_CLOSED) != 0;
  const int nturn = closed ? nk : nk - 2;
  if (nk < 3 || nturn <= 0) return;
  const float4* key = reinterpret_cast<const float4*>(cv.key) + k0;
  auto pt = [&](int i) {
    const float4 q = key[i >= nk ? i - nk : i];
    return make_float2(q.x, q.y);
  };
  // winding sign: the sum of the turn cross products
  float cs = 0.f;
  for (int i = lane; i < nturn; i += 32) {
    const float2 p0 = pt(i), p1 = pt(i + 1), p2 = pt(i + 2);
    const float ax = p1.x - p0.x, ay = p1.y - p0.y, bx = p2.x - p1.x, by = p2.y - p1.y;
    cs += ax * by - ay * bx;
  }
  for (int o = 16; o > 0; o >>= 1) cs += __shfl_xor_sync(0xffffffffu, cs, o);
  const float sgn = cs >= 0.f ? 1.f : -1.f;
  float pen = 0.f;
  for (int i = lane; i < nturn; i += 32) {
    const float2 p0 = pt(i), p1 = pt(i + 1), p2 = pt(i + 2);
    const float ax = p1.x - p0.x, ay = p1.y - p0.y, bx = p2.x - p1.x, by = p2.y - p1.y;
    const float na = sqrtf(ax * ax + ay * ay), nb = sqrtf(bx * bx + by * by);
    if (!(na > 0.f && nb > 0.f)) continue;
    const float cr = ax * by - ay * bx;
    const float inv = 1.f / (na * nb);
    const float sn = cr * inv;
    if (-sgn * sn <= 0.f) continue;
    pen += -sgn * sn;
    if (!dkey) continue;
    const float g = -sgn * lambda;   // dL/dsin
    // dsin/da = (b_y, -b_x)/(|a||b|) - sin a/|a|^2, dsin/db = (-a_y, a_x)/(|a||b|) - sin b/|b|^2
    const float gax = g * (by * inv - sn * ax / (na * na));
    const float gay = g * (-bx * inv - sn * ay / (na * na));
    const float gbx = g * (-ay * inv - sn * bx / (nb * nb));
    const float gby = g * (ax * inv - sn * by / (nb * nb));
    const int i0 = i, i1 = i + 1 >= nk ? i + 1 - nk : i + 1, i2 = i + 2 >= nk ? i + 2 - nk : i + 2;
    float* d0 = dkey + 4 * (long long)(k0 + i0);
    float* d1 = dkey + 4 * (long long)(k0 + i1);
    float* d2 = dkey + 4 * (long long)(k0 + i2);
    atomicAdd(d0 + 0, -gax);
    atomicAdd(d0 + 1, -gay);
    atomicAdd(d1 + 0, gax - gbx);
    atomicAdd(d1 + 1, gay - gby);
    atomicAdd(d2 + 0, gbx);
    atomicAdd(d2 + 1, gby);
  }
  for (int o = 16; o > 0; o >>= 1) pen += __shfl_xor_sync(0xffffffffu, pen, o);
  if (lane == 0 && pen != 0.f) atomicAdd(loss, lambda * pen);
}

struct SeedParams {
  int S, H, W, C, r;
};

// Row pass: rows[pix] = sum of e over the window's columns in the pixel's row.
__global__ void __launch_bounds__(kLiveThreads) k_seed_rows(SeedParams p, const float* __restrict__ image,
                                                            const float* __restrict__ target, float* rows) {
  grid_dep_wait();
  const long long n = (long long)p.S * p.H * p.W;
  for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < n;
       pix += (long long)gridDim.x * blockDim.x) {
    const long long row0 = pix - pix % p.W;
    const int x = int(pix - row0);
    const int x0 = max(0, x - p.r), x1 = min(p.W - 1, x + p.r);
    float v = 0.f;
    for (int xx = x0; xx <= x1; ++xx) {
      for (int ch = 0; ch < p.C; ++ch) {
        const long long i = (row0 + xx) * p.C + ch;
        const float d = image[i] - target[i];
        v = fmaf(d, d, v);
      }
    }
    rows[pix] = v;
  }
}

// Column pass and the packed argmax per scene.
__global__ void __launch_bounds__(kLiveThreads) k_seed_windows(SeedParams p, const float* __restrict__ rows,
                                                               unsigned long long* best) {
  grid_dep_wait();
  const long long hw = (long long)p.H * p.W;
  const long long n = hw * p.S;
  for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < n;
       pix += (long long)gridDim.x * blockDim.x) {
    const int s = int(pix / hw);
    const int rem = int(pix - s * hw);
    const int y = rem / p.W, x = rem - y * p.W;
    const int y0 = max(0, y - p.r), y1 = min(p.H - 1, y + p.r);
    float v = 0.f;
    for (int yy = y0; yy <= y1; ++yy) v += rows[s * hw + (long long)yy * p.W + x];
    const unsigned long long key =
        ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)(0xffffffffu - (unsigned)rem);
    atomicMax(best + s, key);
  }
}

__global__ void k_seed_unpack(int S, int W, const unsigned long long* __restrict__ best, int* seed_xy,
                              float* seed_value) {
  grid_dep_wait();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const unsigned long long k = best[s];
  const int rem = int(0xffffffffu - (unsigned)(k & 0xffffffffull));
  seed_xy[2 * s] = rem % W;
  seed_xy[2 * s + 1] = rem / W;
  if (seed_value) seed_value[s] = __uint_as_float(unsigned(k >> 32));
}

}  // namespace ns

using namespace ns;

extern "C" ns_status ns_udf_mse_loss(const ns_curves* curves, const ns_sample_params* sp,
                                     const ns_raster_params* rp, const ns_capacity* cap, const int32_t* new_curve,
                                     float tau, const float* image, const float* target, float* dL_dimage,
                                     float* loss, void* ws, size_t ws_bytes, void* stream) {
  if (!curves || !sp || !rp || !cap || !new_curve || !image || !target || !loss || !ws) {
    set_error("ns_udf_mse_loss: null argument");
    return NS_ERR_INVALID_ARG;
  }
  if (!(tau > 0.f)) {
    set_error("ns_udf_mse_loss: tau must be > 0");
    return NS_ERR_INVALID_ARG;
  }
  Layout L;
  if (!make_layout(curves, cap, rp, &L)) return NS_ERR_INVALID_ARG;
  if (ws_bytes < L.total) {
    set_error("ns_udf_mse_loss: workspace smaller than ns_workspace_size");
    return NS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  UdfParams up;
  up.S = L.S;
  up.H = L.H;
  up.W = L.W;
  up.C = L.C;
  up.nc = L.nc;
  up.tau = tau;
  up.h = sp->h;
  float* sums = at<float>(ws, L.o_live);
  const CurvePlan* plan = at<const CurvePlan>(ws, L.o_plan);
  const float2* bpts = at<const float2>(ws, L.o_bpts);
  cudaMemsetAsync(sums, 0, sizeof(float) * 4 * (size_t)L.S, s);
  const long long n = (long long)L.S * L.H * L.W;
  const int grid = (int)std::min<long long>((n + kLiveThreads - 1) / kLiveThreads, (long long)num_sms() * 16);
  if (n > 0) {
    NS_LAUNCH(NS_KERNEL_OTHER, k_udf_sums, grid, kLiveThreads, 0, s, up, plan, bpts, new_curve, image, target, sums);
    NS_LAUNCH(NS_KERNEL_OTHER, k_udf_finish, 1, 32, 0, s, up, new_curve, sums, loss);
    if (dL_dimage)
      NS_LAUNCH(NS_KERNEL_OTHER, k_udf_grad, grid, kLiveThreads, 0, s, up, plan, bpts, new_curve, image, target,
                sums, dL_dimage);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("ns_udf_mse_loss: ") + cudaGetErrorString(e));
    return NS_ERR_CUDA;
  }
  return NS_OK;
}

extern "C" ns_status ns_xing_loss(const ns_curves* curves, float lambda, float* loss, float* dkey, void* stream) {
  if (!curves || !loss || !curves->key || !curves->key_offset || !curves->flags || curves->n_curves < 0) {
    set_error("ns_xing_loss: null argument");
    return NS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaMemsetAsync(loss, 0, sizeof(float), s);
  if (curves->n_curves > 0)
    NS_LAUNCH(NS_KERNEL_OTHER, k_xing, (curves->n_curves + 3) / 4, 128, 0, s, *curves, lambda, loss, dkey);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("ns_xing_loss: ") + cudaGetErrorString(e));
    return NS_ERR_CUDA;
  }
  return NS_OK;
}

extern "C" size_t ns_seed_scratch_size(int32_t n_scenes, int32_t height, int32_t width) {
  if (n_scenes < 1 || height < 1 || width < 1) return 0;
  const size_t pix = (size_t)n_scenes * height * width;
  return ((pix * sizeof(float) + 255) & ~size_t(255)) + sizeof(unsigned long long) * (size_t)n_scenes;
}

extern "C" ns_status ns_seed_windows(const float* image, const float* target, int32_t n_scenes, int32_t height,
                                     int32_t width, int32_t channels, int32_t radius, void* scratch,
                                     size_t scratch_bytes, int32_t* seed_xy, float* seed_value, void* stream) {
  if (!image || !target || !scratch || !seed_xy) {
    set_error("ns_seed_windows: null argument");
    return NS_ERR_INVALID_ARG;
  }
  if (n_scenes < 1 || height < 1 || width < 1 || channels < 1 || channels > 4 || radius < 0) {
    set_error("ns_seed_windows: sizes must be positive, channels 1..4, radius >= 0");
    return NS_ERR_INVALID_ARG;
  }
  const size_t need = ns_seed_scratch_size(n_scenes, height, width);
  if (scratch_bytes < need) {
    set_error("ns_seed_windows: scratch smaller than ns_seed_scratch_size");
    return NS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SeedParams p;
  p.S = n_scenes;
  p.H = height;
  p.W = width;
  p.C = channels;
  p.r = radius;
  const size_t pix = (size_t)n_scenes * height * width;
  float* rows = static_cast<float*>(scratch);
  unsigned long long* best =
      reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + ((pix * sizeof(float) + 255) & ~size_t(255)));
  cudaMemsetAsync(best, 0, sizeof(unsigned long long) * (size_t)n_scenes, s);
  const int grid = (int)std::min<long long>(((long long)pix + kLiveThreads - 1) / kLiveThreads,
                                            (long long)num_sms() * 16);
  NS_LAUNCH(NS_KERNEL_OTHER, k_seed_rows, grid, kLiveThreads, 0, s, p, image, target, rows);
  NS_LAUNCH(NS_KERNEL_OTHER, k_seed_windows, grid, kLiveThreads, 0, s, p, rows, best);
  NS_LAUNCH(NS_KERNEL_OTHER, k_seed_unpack, (n_scenes + 127) / 128, 128, 0, s, n_scenes, width, best, seed_xy,
            seed_value);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("ns_seed_windows: ") + cudaGetErrorString(e));
    return NS_ERR_CUDA;
  }
  return NS_OK;
}
