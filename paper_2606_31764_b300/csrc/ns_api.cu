// Host side of the C ABI: defaults, workspace layout, status, the L2 loss,
// the Adam step and the error channel.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>

#include "ns_internal.cuh"

namespace ns {

static thread_local std::string g_error;
static thread_local unsigned long long g_launches = 0;
// Armed profiling records: one-shot (kernel, start event, stop event) entries.
struct ProfArm {
  int kernel;
  cudaEvent_t start, stop;
  bool started;
};
constexpr int kMaxArms = 32;
static thread_local ProfArm g_arms[kMaxArms];
static thread_local int g_n_arms = 0;

void set_error(const std::string& msg) { g_error = msg; }

static void record_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s, &cs);
  if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else cudaEventRecord(e, s);
}

void before_launch(int kernel_id, cudaStream_t s) {
  ++g_launches;
  for (int i = 0; i < g_n_arms; ++i)
    if (g_arms[i].kernel == kernel_id && !g_arms[i].started) {
      record_event(g_arms[i].start, s);
      g_arms[i].started = true;
      break;
    }
}

void after_launch(int kernel_id, cudaStream_t s) {
  for (int i = 0; i < g_n_arms; ++i)
    if (g_arms[i].kernel == kernel_id && g_arms[i].started) {
      record_event(g_arms[i].stop, s);
      g_arms[i] = g_arms[--g_n_arms];   // one shot: drop the entry
      break;
    }
}

// A profiled range with no launch in it (a stage that had nothing to do):
// its two events are recorded back to back, and no launch is counted.
void empty_range(int kernel_id, cudaStream_t s) {
  for (int i = 0; i < g_n_arms; ++i)
    if (g_arms[i].kernel == kernel_id && !g_arms[i].started) {
      record_event(g_arms[i].start, s);
      record_event(g_arms[i].stop, s);
      g_arms[i] = g_arms[--g_n_arms];
      break;
    }
}

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("NS_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

int num_sms() {
  static thread_local int cached_dev = -1, cached_n = 148;
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return cached_n;
  if (dev == cached_dev) return cached_n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return cached_n;
  cached_dev = dev;
  cached_n = n;
  return n;
}

static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

bool make_layout(const ns_curves* c, const ns_capacity* cap, const ns_raster_params* rp, Layout* L) {
  if (!c || !cap || !rp) {
    set_error("null curves, capacity or raster parameters");
    return false;
  }
  if (c->n_scenes < 1 || c->n_curves < 0 || c->n_keys < 0 || c->n_taus < 0 || c->height < 1 || c->width < 1 ||
      (c->channels != 1 && c->channels != 3)) {
    set_error("invalid sizes: need n_scenes >= 1, height, width >= 1, channels 1 or 3");
    return false;
  }
  if (c->n_curves > 0 && (!c->degree || !c->flags || !c->key_offset || !c->tau_offset || !c->key || !c->tau ||
                          !c->color)) {
    set_error("curve tables must be non-null");
    return false;
  }
  if (c->n_scenes > 1 && !c->scene_curve_offset) {
    set_error("scene_curve_offset is required with more than one scene");
    return false;
  }
  if (cap->gaussians < 0 || cap->pairs < 0 || cap->boundary < 0 || cap->gaussians >= (1LL << 31) ||
      cap->pairs >= (1LL << 31) || cap->boundary >= (1LL << 31)) {
    set_error("capacities must lie in [0, 2^31)");
    return false;
  }
  if (rp->tile != 8 && rp->tile != 16 && rp->tile != 32) {
    set_error("tile must be 8, 16 or 32");
    return false;
  }
  L->S = c->n_scenes;
  L->H = c->height;
  L->W = c->width;
  L->C = c->channels;
  L->tile = rp->tile;
  L->tiles_x = (c->width + rp->tile - 1) / rp->tile;
  L->tiles_y = (c->height + rp->tile - 1) / rp->tile;
  const long long nt = (long long)L->S * L->tiles_x * L->tiles_y;
  if (nt >= (1LL << 31) || L->tiles_x > 32767 || L->tiles_y > 32767) {
    set_error("too many tiles (at most 32767 per image side and 2^31 in all)");
    return false;
  }
  L->n_tiles = int(nt);
  L->n_pix = (int64_t)L->S * L->H * L->W;
  L->nc = c->n_curves;
  L->nk = c->n_keys;
  L->nt = c->n_taus;
  L->gcap = cap->gaussians;
  L->pcap = cap->pairs;
  L->bcap = cap->boundary;
  L->bin_blocks = (L->gcap + kBinItems - 1) / kBinItems;
  L->sort_blocks = (L->pcap + kSortItems - 1) / kSortItems;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t r = o;
    o = align_up(o + bytes);
    return r;
  };
  const size_t nkn = (size_t)L->nt + (size_t)kKnotPad * L->nc;
  L->o_state = take(sizeof(DevState));
  L->o_plan = take(sizeof(CurvePlan) * (size_t)L->nc);
  L->o_knots = take(sizeof(float) * nkn);
  L->o_dknots = take(sizeof(float) * nkn);
  L->o_order = take(sizeof(int) * (size_t)L->nc);
  L->o_curve_scene = take(sizeof(int) * (size_t)L->nc);
  L->o_bpts = take(sizeof(float2) * (size_t)L->bcap);
  L->o_dbpts = take(sizeof(float2) * (size_t)L->bcap);
  L->o_bcurve = take(sizeof(int) * (size_t)L->bcap);
  L->o_cbox = take(sizeof(float4) * (size_t)L->bcap);   // at the index of each cluster's first point
  L->o_bloc = take(sizeof(float4) * (size_t)L->bcap);
  L->o_glo = take(sizeof(float2) * (size_t)L->nc);
  L->o_knots_lo = take(sizeof(float) * nkn);
  L->o_krcp = take(sizeof(float2) * kMaxP * nkn);
  L->o_forms = take(sizeof(float) * kFormStride * nkn);   // span Taylor forms, one row per knot slot
  L->o_boffs = take(sizeof(int) * (size_t)L->nc);          // first boundary point of each curve, packed
  L->o_lbox = take(sizeof(int4) * (size_t)L->nc);
  L->o_bmix = take(sizeof(int) * (size_t)(L->bin_blocks + 1));
  // contour tasks cover a curve's samples in chunks of kChunk, fill tasks its
  // grid in T x T tiles, T = 8 or 16 (at most (nx ny + (T - 1)(nx + ny) +
  // (T - 1)^2) / T^2 of them): within the Gaussian capacity this table holds
  // them all (past it the task -> curve search takes over)
  L->tcap = L->gcap / kChunk + L->gcap / 64 + L->gcap / 8 + 2LL * L->nc + 1;
  L->o_tasks = take(sizeof(int) * (size_t)L->tcap);
  L->sample_total = o;   // everything above depends on the curves and capacities only
  L->o_bsum = take(sizeof(int) * (size_t)(L->bin_blocks + 1));
  L->o_k0 = take(sizeof(uint32_t) * (size_t)L->pcap);
  L->o_v0 = take(sizeof(uint32_t) * (size_t)L->pcap);
  L->o_k1 = take(sizeof(uint32_t) * (size_t)L->pcap);
  L->o_v1 = take(sizeof(uint32_t) * (size_t)L->pcap);
  L->o_hist = take(sizeof(uint32_t) * 256 * (size_t)(L->sort_blocks + kMaxRadixPasses));   // + digit totals
  L->o_ranges = take(sizeof(int2) * (size_t)L->n_tiles);
  L->o_T = take(sizeof(float) * (size_t)L->n_pix);
  L->o_nlast = take(sizeof(int) * (size_t)L->n_pix);
  L->o_nsub = take(sizeof(int) * (size_t)L->n_pix);
  // fill layers: per curve, the grid run of each tile column and row
  L->o_lruns = take(sizeof(int2) * (size_t)L->nc * (size_t)(L->tiles_x + L->tiles_y));
  L->o_lconst = take(sizeof(float4) * 3 * (size_t)L->nc);   // per layer {X0, Y0, xoff, yoff}, {sigma, ncoef, nx, ny}, {h, 1/h, R, 0}
  L->o_bflag = take(sizeof(int) * (size_t)(L->bin_blocks + 1));
  L->o_lcount = take(sizeof(int) * (size_t)L->nc);
  L->o_lmin = take(sizeof(int2) * (size_t)L->nc);   // per layer: smallest live grid column and row
  L->o_lmax = take(sizeof(int2) * (size_t)L->nc);   // largest
  L->o_dgauss = take(sizeof(float) * 12 * (size_t)L->gcap);   // 8 per Gaussian, 12 when tangent-aligned
  L->o_prep = take(sizeof(float4) * (size_t)L->gcap);
  L->o_prep2 = take(sizeof(float2) * (size_t)L->gcap);
  L->o_reach = take(sizeof(float2) * (size_t)L->gcap);
  L->o_live = take(sizeof(float) * 4 * (size_t)L->S);
  L->total = o;
  return true;
}

int sorted_buffer(const Layout& L);

// Resets the status word and counters; with nurbs_sample also zeroes the
// curve order (in range even if the scene offsets are bad) and the Gaussian
// count (in this launch instead of a memset each).
__global__ void k_reset_state(DevState* st, int* order, int n_order, int* count_out) {
  grid_dep_wait();
  for (int i = threadIdx.x; i < n_order; i += blockDim.x) order[i] = 0;
  if (threadIdx.x != 0) return;
  if (count_out) *count_out = 0;
  st->status = 0;
  st->bad_curve = -1;
  st->n_chunks = 0;
  st->n_ctasks = 0;
  st->g_total = st->b_total = st->pair_total = st->culled = 0;
  st->g_count = st->pair_count = st->b_count = 0;
  st->blend_evals = st->blend_bwd_evals = st->blend_contribs = 0;
  st->blend_visits = st->blend_bwd_visits = 0;
  st->cull_thr = -1.f;
  st->culled_s = 0;
}

void launch_reset_state(DevState* st, cudaStream_t s, int* order, int n_order, int* count_out) {
  NS_LAUNCH(NS_KERNEL_OTHER, k_reset_state, 1, n_order > 0 ? 256 : 1, 0, s, st, order, n_order, count_out);
}

__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ a, const float* __restrict__ b, long long n,
                                             float* __restrict__ grad, float* loss) {
  grid_dep_wait();
  __shared__ float red[8];
  const float scale = 2.f / float(n);
  float acc = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long head = 0;   // values handled four at a time
  if (((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(grad)) & 15) == 0) {
    const long long n4 = n >> 2;
    const float4* a4 = reinterpret_cast<const float4*>(a);
    const float4* b4 = reinterpret_cast<const float4*>(b);
    float4* g4 = reinterpret_cast<float4*>(grad);
    for (long long i = t0; i < n4; i += stride) {
      const float4 x = a4[i], y = b4[i];
      const float d0 = x.x - y.x, d1 = x.y - y.y, d2 = x.z - y.z, d3 = x.w - y.w;
      acc = fmaf(d0, d0, acc);
      acc = fmaf(d1, d1, acc);
      acc = fmaf(d2, d2, acc);
      acc = fmaf(d3, d3, acc);
      if (grad) g4[i] = make_float4(scale * d0, scale * d1, scale * d2, scale * d3);
    }
    head = n4 << 2;
  }
  for (long long i = head + t0; i < n; i += stride) {
    const float d = a[i] - b[i];
    acc = fmaf(d, d, acc);
    if (grad) grad[i] = scale * d;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < 8; ++w) s += red[w];
    atomicAdd(loss, s / float(n));
  }
}

struct Clamp4 {
  float lo[4], hi[4], lr[4];   // per component of the group: clamp bounds and learning rate
};

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float b1, float b2, float eps, float c1, float c2, Clamp4 cl, int group) {
  grid_dep_wait();
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / c1, vh = vi / c2;
    const int j = int(i % group);
    const float x = p[i] - cl.lr[j] * mh / (sqrtf(vh) + eps);
    p[i] = fminf(fmaxf(x, cl.lo[j]), cl.hi[j]);
  }
}

}  // namespace ns

using namespace ns;

extern "C" {

ns_sample_params ns_default_sample_params(void) {
  ns_sample_params p;
  p.delta_c = 10.f;   // Table S1
  p.rho = 2.f;
  p.delta_b = 0.5f;
  p.h = 1.f;
  p.eta = 1.5f;
  p.gamma = 5.f;
  p.pad_frac = 0.1f;  // padding "proportional to the extent": 10 %
  p.kappa = 4;
  p.nl_mult = 3;
  p.fill_rule = 0;
  p.fill_cull = 0.f;
  p.contour_mode = 0;  // isotropic contour Gaussians (Eq. 5)
  p.fill_tile = 0;     // 16 x 16 fill tiles
  return p;
}

ns_raster_params ns_default_raster_params(void) {
  ns_raster_params r;
  r.tile = 16;
  r.k_sigma = 3.5f;
  r.alpha_min = 1.f / 255.f;
  r.alpha_max = 0.99f;
  r.t_min = 1e-4f;
  r.bg[0] = r.bg[1] = r.bg[2] = 1.f;
  r.ppt_fwd = 0;
  r.ppt_bwd = 0;
  r.fill_layers = 0;
  return r;
}

size_t ns_workspace_size(const ns_curves* curves, const ns_capacity* cap, const ns_raster_params* raster) {
  Layout L;
  if (!make_layout(curves, cap, raster, &L)) return 0;
  return L.total;
}

float ns_grid_step(int32_t t, int32_t T, float h_max, float h_min, float t_b, float t_e) {
  const double f = T > 0 ? double(t) / double(T) : 1.0;
  if (f <= t_b) return h_max;
  if (f >= t_e) return h_min;
  const double phi = (f - t_b) / (double(t_e) - double(t_b));
  return float(h_max + (double(h_min) - h_max) * (1.0 + cos(3.14159265358979323846 * (1.0 - phi))) * 0.5);
}

ns_status ns_poll_status(void* ws, ns_report* r, void* stream) {
  if (!ws || !r) {
    set_error("ns_poll_status: null argument");
    return NS_ERR_INVALID_ARG;
  }
  DevState st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&st, ws, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_error(std::string("ns_poll_status: ") + cudaGetErrorString(cudaGetLastError()));
    return NS_ERR_CUDA;
  }
  r->status = st.status;
  r->bad_curve = st.bad_curve;
  r->gaussians = (int64_t)st.g_total;
  r->pairs = (int64_t)st.pair_total;
  r->boundary = (int64_t)st.b_total;
  r->fill_culled = (int64_t)st.culled;
  r->blend_evals = (int64_t)st.blend_evals;
  r->blend_bwd_evals = (int64_t)st.blend_bwd_evals;
  r->blend_contribs = (int64_t)st.blend_contribs;
  r->blend_visits = (int64_t)st.blend_visits;
  r->blend_bwd_visits = (int64_t)st.blend_bwd_visits;
  return NS_OK;
}

ns_status ns_clear_status(void* ws, void* stream) {
  if (!ws) {
    set_error("ns_clear_status: null workspace");
    return NS_ERR_INVALID_ARG;
  }
  NS_LAUNCH(NS_KERNEL_OTHER, k_reset_state, 1, 1, 0, static_cast<cudaStream_t>(stream), static_cast<DevState*>(ws),
            static_cast<int*>(nullptr), 0, static_cast<int*>(nullptr));
  return cudaGetLastError() == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

ns_status ns_mse_loss(const float* image, const float* target, int64_t n, float* dL, float* loss, void* stream) {
  if (!image || !target || !loss || n <= 0) {
    set_error("ns_mse_loss: null argument or n <= 0");
    return NS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaMemsetAsync(loss, 0, sizeof(float), s);
  const long long blocks = (n / 4 + 255) / 256 + 1;
  const int grid = int(blocks < num_sms() * 8 ? blocks : num_sms() * 8);
  NS_LAUNCH(NS_KERNEL_MSE, k_mse, grid, 256, 0, s, image, target, n, dL, loss);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("ns_mse_loss: ") + cudaGetErrorString(e));
    return NS_ERR_CUDA;
  }
  return NS_OK;
}

ns_status ns_adam_step(float* param, const float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                       float beta2, float eps, int32_t step, const float* lo, const float* hi, int32_t group,
                       const float* lr_scale, void* stream) {
  if (!param || !grad || !m || !v || n < 0 || step < 1 || !lo || !hi || group < 1 || group > 4) {
    set_error("ns_adam_step: invalid argument");
    return NS_ERR_INVALID_ARG;
  }
  Clamp4 cl;
  for (int j = 0; j < 4; ++j) {
    cl.lo[j] = j < group ? lo[j] : -INFINITY;
    cl.hi[j] = j < group ? hi[j] : INFINITY;
    cl.lr[j] = lr * (lr_scale && j < group ? lr_scale[j] : 1.f);
    if (!(cl.lo[j] <= cl.hi[j])) {
      set_error("ns_adam_step: lo > hi");
      return NS_ERR_INVALID_ARG;
    }
  }
  if (n == 0) return NS_OK;
  const float c1 = 1.f - powf(beta1, float(step));
  const float c2 = 1.f - powf(beta2, float(step));
  const long long blocks = (n + 255) / 256;
  const int grid = int(blocks < num_sms() * 8 ? blocks : num_sms() * 8);
  NS_LAUNCH(NS_KERNEL_ADAM, k_adam, grid, 256, 0, static_cast<cudaStream_t>(stream), param, grad, m, v, n, beta1,
            beta2, eps, c1, c2, cl, group);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("ns_adam_step: ") + cudaGetErrorString(e));
    return NS_ERR_CUDA;
  }
  return NS_OK;
}

ns_status ns_workspace_copy(void* ws, const ns_curves* curves, const ns_capacity* cap, const ns_raster_params* rp,
                            int32_t which, void* dst, size_t bytes, void* stream) {
  Layout L;
  if (!ws || !dst || !make_layout(curves, cap, rp, &L)) {
    if (!ws || !dst) set_error("ns_workspace_copy: null argument");
    return NS_ERR_INVALID_ARG;
  }
  const int sb = sorted_buffer(L);
  size_t off = 0, avail = 0;
  switch (which) {
    case 0: off = sb ? L.o_k1 : L.o_k0; avail = 4 * (size_t)L.pcap; break;
    case 1: off = sb ? L.o_v1 : L.o_v0; avail = 4 * (size_t)L.pcap; break;
    case 2: off = L.o_ranges; avail = 8 * (size_t)L.n_tiles; break;
    case 3: off = L.o_plan; avail = sizeof(CurvePlan) * (size_t)L.nc; break;
    case 4: off = L.o_bpts; avail = 8 * (size_t)L.bcap; break;
    case 5: off = L.o_T; avail = 4 * (size_t)L.n_pix; break;
    case 6: off = L.o_nlast; avail = 4 * (size_t)L.n_pix; break;
    default:
      set_error("ns_workspace_copy: unknown array");
      return NS_ERR_INVALID_ARG;
  }
  if (bytes > avail) {
    set_error("ns_workspace_copy: more bytes than the array holds");
    return NS_ERR_INVALID_ARG;
  }
  if (bytes && cudaMemcpyAsync(dst, static_cast<char*>(ws) + off, bytes, cudaMemcpyDeviceToDevice,
                               static_cast<cudaStream_t>(stream)) != cudaSuccess) {
    set_error("ns_workspace_copy: copy failed");
    return NS_ERR_CUDA;
  }
  return NS_OK;
}

ns_status ns_profile_next_launch(int32_t kernel_id, void* start, void* stop) {
  if (kernel_id == 0) {
    g_n_arms = 0;
    return NS_OK;
  }
  if (!start || !stop) {
    set_error("ns_profile_next_launch: events required");
    return NS_ERR_INVALID_ARG;
  }
  if (g_n_arms >= kMaxArms) {
    set_error("ns_profile_next_launch: too many armed launches");
    return NS_ERR_INVALID_ARG;
  }
  g_arms[g_n_arms++] = ProfArm{kernel_id, static_cast<cudaEvent_t>(start), static_cast<cudaEvent_t>(stop), false};
  return NS_OK;
}

uint64_t ns_launch_count(void) { return g_launches; }

const char* ns_last_error(void) { return g_error.c_str(); }

}  // extern "C"
