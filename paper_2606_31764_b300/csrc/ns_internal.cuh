// Internal definitions shared by the library's translation units: workspace
// layout, device state, per-curve plan records and the span-local NURBS
// evaluator (forward and reverse mode).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "nurbs_splat.h"

namespace ns {

constexpr int kMaxP = NS_MAX_DEGREE;
constexpr int kChunk = 256;          // Gaussians per sampling / chain task (one block)
constexpr int kFillTileMax = 16;     // a fill task: a T x T tile of its curve's grid, T = 8 or 16
constexpr int kBinItems = 2048;      // Gaussians per binning block (256 threads x 8)
constexpr int kSortItems = 4096;     // pairs per radix-sort block (256 threads x 16)
constexpr int kSortThreads = 256;
constexpr int kFormStride = 20;      // floats per span Taylor form row (19 used at degree 5)
constexpr int kMaxRadixPasses = 4;   // 32 tile bits at 8 bits per pass
constexpr int kKnotPad = 2 * kMaxP + 1;  // knots per curve = intervals + 2p + 1

enum CurveKind : int { kNone = 0, kOpen = 1, kClosedStroke = 2, kFill = 3 };

// aux code of a fill Gaussian whose grid point lies so deep inside that its
// sigmoid is exactly 1 in FP32: no nearest segment is recorded (none is needed)
constexpr int kAuxDeep = 0x7fffffff;
// aux code of a fill Gaussian provably outside with opacity below the cull
// threshold (written with opacity 0; it bins to no tile)
constexpr int kAuxFar = int(0x80000000u);

// Device-side status and counters, at the start of the workspace.
struct DevState {
  int status;          // ns_status, first error wins
  int bad_curve;
  int n_chunks;        // fill tasks of the current sample (numbered first)
  int n_ctasks;        // contour tasks (numbered after the fill tasks)
  int sorted_buf;      // which pair buffer holds the sorted result
  unsigned long long g_total;     // Gaussians needed
  unsigned long long b_total;     // boundary points needed
  unsigned long long pair_total;  // pairs needed
  unsigned long long culled;      // fill Gaussians with opacity < alpha_min
  int g_count;         // min(g_total, capacity)
  int pair_count;      // min(pair_total, capacity)
  int b_count;
  int pad[4];
  unsigned long long blend_evals;      // alpha evaluations of the last forward blend
  unsigned long long blend_bwd_evals;  // alpha evaluations of the last backward blend
  unsigned long long blend_contribs;   // composited (pixel, Gaussian) pairs of the last forward blend
  unsigned long long blend_visits;     // (pixel, list entry) pairs walked by the last forward blend
  unsigned long long blend_bwd_visits; // the same for the last backward blend
  // what nurbs_sample knows of its fill Gaussians for a given alpha_min (its
  // fill_cull): the culled count, and (in the workspace) each curve's box of
  // live grid points; the binning uses them when its alpha_min is the same
  float cull_thr;                      // the threshold they were counted for (-1: none)
  int sdf_next;                        // the next fill task k_fill_sdf hands out (k_boundary_box resets it)
  unsigned long long culled_s;         // fill Gaussians with opacity below cull_thr (sigma > 0)
};

// One curve's sampling plan (written by the planning kernels).
struct CurvePlan {
  float L, a, b, x0, y0;   // arc length, domain [a, b], fill grid origin
  int kind;                // CurveKind
  int M;                   // contour samples (open/closed) or boundary points (fill)
  int count;               // Gaussians emitted
  int nx, ny;              // fill grid
  int g_off;               // first Gaussian (front-to-back order)
  int b_off;               // first boundary point
  int chunk_off;           // first task of this curve's kind (fill tasks and contour tasks are numbered separately)
  int scene;
  int pad[1];
  float h;                 // fill grid step (0 for strokes)
};
static_assert(sizeof(CurvePlan) == 64, "plan record is one 64-byte line");

struct Layout {
  int S = 0, H = 0, W = 0, C = 0, tile = 16, tiles_x = 0, tiles_y = 0, n_tiles = 0;
  int64_t n_pix = 0;
  int nc = 0, nk = 0, nt = 0;
  int64_t gcap = 0, pcap = 0, bcap = 0;
  int64_t bin_blocks = 0, sort_blocks = 0;
  size_t o_state = 0, o_plan = 0, o_knots = 0, o_dknots = 0, o_bpts = 0, o_dbpts = 0, o_bsum = 0,
         o_k0 = 0, o_v0 = 0, o_k1 = 0, o_v1 = 0, o_hist = 0, o_ranges = 0, o_T = 0, o_nlast = 0, o_nsub = 0, o_lruns = 0, o_lconst = 0, o_lmin = 0, o_lmax = 0,
         o_dgauss = 0, o_curve_scene = 0, o_order = 0, o_prep = 0, o_prep2 = 0, o_reach = 0, o_live = 0,
         total = 0;
  size_t sample_total = 0;   // bytes of the prefix nurbs_sample uses (independent of the raster settings)
  size_t o_tasks = 0;        // task -> curve table (fill tasks first, then contour tasks)
  size_t o_bcurve = 0;       // boundary point -> curve
  size_t o_cbox = 0;         // bounding box of each 8-segment cluster of a boundary polyline
  size_t o_bloc = 0;         // boundary points relative to their curve's fill grid origin, {x_hi, y_hi, x_lo, y_lo}
  size_t o_glo = 0;          // per curve: the low parts {x0_lo, y0_lo} of the fill grid origin (plan x0, y0 = high parts)
  size_t o_knots_lo = 0;     // low parts of the knot vectors (knots = their high parts, the exact sums rounded)
  size_t o_lbox = 0;         // per curve: {min column, min row, max column, max row} of live fill grid points (nurbs_sample)
  size_t o_bmix = 0;         // per binning block: 1 if a Gaussian of a stroke (not a filled curve) lies in it (nurbs_sample)
  size_t o_bflag = 0;        // per binning block: 1 if it holds a Gaussian that is not a fill layer's (splat_forward)
  size_t o_lcount = 0;       // per curve: tile pairs of its fill layer (splat_forward)
  size_t o_krcp = 0;         // per knot slot k and width j = 1..kMaxP: 1 / (U[k + j] - U[k]) as {hi, lo} (filled curves)
  int64_t tcap = 0;          // entries of that table
  size_t o_boffs = 0;        // per curve: its first boundary point (plan b_off, packed for searches)
  size_t o_forms = 0;        // per knot slot: the Taylor form {m, A[0..p][3]} of the span it starts (20 floats)
};

// Host helpers (ns_api.cu).
void set_error(const std::string& msg);
bool make_layout(const ns_curves* c, const ns_capacity* cap, const ns_raster_params* rp, Layout* L);
int num_sms();
void launch_reset_state(DevState* st, cudaStream_t s, int* order, int n_order, int* count_out);

// Launch bookkeeping: counts launches and fires the armed profiling events.
void before_launch(int kernel_id, cudaStream_t s);
void after_launch(int kernel_id, cudaStream_t s);
void empty_range(int kernel_id, cudaStream_t s);

// Programmatic dependent launch.  The library's kernels are launched with
// programmatic stream serialization: a kernel's launch may overlap the end of
// the kernel before it in the stream (or graph), and every kernel begins with
// grid_dep_wait(), which returns once that kernel has completed and its
// writes are visible.  So the order of memory effects is that of a plain
// stream; what overlaps is the launch and the start of the next kernel's
// blocks with the last blocks of this one.  A kernel launched without the
// attribute returns from the wait at once.  The environment variable NS_PDL=0
// launches without it.
bool pdl_enabled();
template <typename... KArgs, typename... Args>
inline void launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                          Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}
#define NS_LAUNCH(id, kernel, grid, block, smem, stream, ...)                 \
  do {                                                                       \
    ::ns::before_launch(id, stream);                                         \
    ::ns::launch_kernel(kernel, grid, block, smem, stream, __VA_ARGS__);     \
    ::ns::after_launch(id, stream);                                          \
  } while (0)

template <typename T>
inline T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

// ---------------------------------------------------------------------------
// device helpers

// The first statement of every kernel (see launch_kernel): wait for the
// kernel before, then allow the next kernel to launch.  Its blocks take SM
// slots only as this grid's blocks finish (the trigger fires once every block
// of this grid has run it) and wait in their own grid_dep_wait() until this
// grid has completed.
__device__ __forceinline__ void grid_dep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);
}

__device__ __forceinline__ void raise_status(DevState* st, int code) {
  atomicCAS(&st->status, 0, code);
}

__device__ __forceinline__ int cp_to_key(int cp, int p, bool closed, int nk) {
  if (!closed) return cp;
  int k = cp - (p + 1) / 2;
  k %= nk;
  return k < 0 ? k + nk : k;
}

// Largest span i in [p, n] with U[i] <= u and U[i] < U[i+1] (a non-empty
// span; at the right end of the domain and at repeated knots the last
// non-empty span below u is used).
__device__ __forceinline__ int find_span(const float* U, int p, int n, float u) {
  if (!(u >= U[p])) return p;
  int lo = p, hi = n;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (U[mid] <= u) lo = mid; else hi = mid - 1;
  }
  while (lo > p && !(U[lo] < U[lo + 1])) --lo;
  return lo;
}

// Span-local Cox-de Boor triangle for degree P at parameter u in span i.
// lev[j][r] keeps N_{i-j+r, j} for j < P (needed by the reverse sweep and the
// derivative), N[r] = N_{i-P+r, P}.  left[j] = u - U[i+1-j], right[j] = U[i+j] - u.
template <int P>
struct Tri {
  float lev[P][P];
  float N[P + 1];
  float left[P + 1], right[P + 1];
};

template <int P>
__device__ __forceinline__ void basis_fwd(const float* __restrict__ U, int i, float u, Tri<P>& t) {
  float N[P + 1];
  N[0] = 1.f;
#pragma unroll
  for (int j = 1; j <= P; ++j) {
    t.left[j] = u - U[i + 1 - j];
    t.right[j] = U[i + j] - u;
#pragma unroll
    for (int r = 0; r < j; ++r) t.lev[j - 1][r] = N[r];
    float saved = 0.f;
#pragma unroll
    for (int r = 0; r < j; ++r) {
      const float temp = N[r] / (t.right[r + 1] + t.left[j - r]);
      N[r] = saved + t.right[r + 1] * temp;
      saved = t.left[j - r] * temp;
    }
    N[j] = saved;
  }
#pragma unroll
  for (int r = 0; r <= P; ++r) t.N[r] = N[r];
}

// First derivatives N'_{i-P+r, P}, r = 0..P, from level P-1 of the triangle.
template <int P>
__device__ __forceinline__ void basis_deriv(const Tri<P>& t, float* dN) {
  float tmp[P + 1];
#pragma unroll
  for (int r = 0; r < P; ++r) tmp[r] = t.lev[P - 1][r] / (t.right[r + 1] + t.left[P - r]);
#pragma unroll
  for (int r = 0; r <= P; ++r) {
    const float a = r > 0 ? tmp[r - 1] : 0.f;
    const float b = r < P ? tmp[r] : 0.f;
    dN[r] = float(P) * (a - b);
  }
}

// Reverse sweep through the triangle.  Given g[r] = dL/dN_{i-P+r,P}, adds
// dL/du to *du and dL/dU[k] to dU[k - (i-P+1)] for the 2P local knots.
// Level j forms N^{(j)}[r] = beta_r x_r + alpha_{r-1} x_{r-1}, x = level j-1,
// alpha_r = (u - U_lo)/(U_hi - U_lo), beta_r = 1 - alpha_r,
// lo = i+r+1-j, hi = i+r+1.
template <int P>
__device__ __forceinline__ void basis_bwd(const Tri<P>& t, const float* gN, float* du, float* dU) {
  float g[P + 1];
#pragma unroll
  for (int r = 0; r <= P; ++r) g[r] = gN[r];
#pragma unroll
  for (int j = P; j >= 1; --j) {
    float gp[P];
#pragma unroll
    for (int r = 0; r < j; ++r) {
      const float x = t.lev[j - 1][r];
      const float D = t.right[r + 1] + t.left[j - r];
      const float inv = 1.f / D;
      const float al = t.left[j - r] * inv;
      const float be = t.right[r + 1] * inv;
      gp[r] = be * g[r] + al * g[r + 1];
      const float dal = x * (g[r + 1] - g[r]);
      *du += dal * inv;
      dU[r + P - j] += dal * (al - 1.f) * inv;
      dU[r + P] -= dal * al * inv;
    }
#pragma unroll
    for (int r = 0; r < j; ++r) g[r] = gp[r];
  }
}

// Per-curve constants resolved from the input tables.
struct CurveRef {
  int p, nk, ntau, key0, knot0, n;  // n: last control point index
  bool closed, filled;
};

__device__ __forceinline__ CurveRef curve_ref(const ns_curves& cv, int c) {
  CurveRef r;
  r.p = cv.degree[c];
  const int fl = cv.flags[c];
  r.closed = (fl & NS_CLOSED) != 0;
  r.filled = (fl & NS_FILLED) != 0;
  r.key0 = cv.key_offset[c];
  r.nk = cv.key_offset[c + 1] - r.key0;
  const int t0 = cv.tau_offset[c];
  r.ntau = cv.tau_offset[c + 1] - t0;
  r.knot0 = t0 + kKnotPad * c;
  r.n = r.closed ? r.nk + r.p - 1 : r.nk - 1;
  return r;
}

// C(u) = S/W (Eq. 1) in span i with its triangle; optionally C'(u) (Eq. 2).
template <int P>
struct Eval {
  Tri<P> t;
  float4 cp[P + 1];   // {x, y, s, w} of the span's control points
  float S[3], W, C[3];
};

template <int P>
__device__ __forceinline__ void eval_curve(const float4* __restrict__ key, const CurveRef& cr,
                                           const float* __restrict__ U, int i, float u, Eval<P>& e) {
  basis_fwd<P>(U, i, u, e.t);
  e.S[0] = e.S[1] = e.S[2] = 0.f;
  e.W = 0.f;
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    const int k = cp_to_key(i - P + l, P, cr.closed, cr.nk);
    const float4 q = key[cr.key0 + k];   // key may point to shared or global memory: plain load
    e.cp[l] = q;
    const float nw = e.t.N[l] * q.w;
    e.S[0] = fmaf(nw, q.x, e.S[0]);
    e.S[1] = fmaf(nw, q.y, e.S[1]);
    e.S[2] = fmaf(nw, q.z, e.S[2]);
    e.W += nw;
  }
  const float iw = 1.f / e.W;
  e.C[0] = e.S[0] * iw;
  e.C[1] = e.S[1] * iw;
  e.C[2] = e.S[2] * iw;
}

// Reverse of C = S/W at one evaluated point: given gC = dL/dC (x, y, s), adds
// dL/d{x, y, s, w} of the span's control points to dcp[l], dL/dU of its 2P
// knots to dkn (as basis_bwd) and returns dL/du in *du.  Without KNOTS (knot
// intervals frozen) the reverse sweep of the triangle, which only feeds the
// knot and parameter gradients, is skipped and *du is 0.
template <int P, bool KNOTS = true>
__device__ __forceinline__ void curve_point_adjoint(const Eval<P>& e, const float gC[3], float dcp[P + 1][4],
                                                    float dkn[2 * P], float* du) {
  const float iw = 1.f / e.W;
  float gN[P + 1];
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    const float4 q = e.cp[l];
    const float R = e.t.N[l] * q.w * iw;              // rational basis N w / W
    const float proj = gC[0] * (q.x - e.C[0]) + gC[1] * (q.y - e.C[1]) + gC[2] * (q.z - e.C[2]);
    gN[l] = q.w * proj * iw;                            // dL/dN_l
    dcp[l][0] += gC[0] * R;
    dcp[l][1] += gC[1] * R;
    dcp[l][2] += gC[2] * R;
    dcp[l][3] += e.t.N[l] * proj * iw;
  }
  float d = 0.f;
  if constexpr (KNOTS) basis_bwd<P>(e.t, gN, &d, dkn);
  *du = d;
}

// Reverse sweep of the span triangle with adjoints entering at every level:
// gTop[r] = dL/dN_{i-P+r,P}, gLow[d][r] = dL/dN_{i-d+r,d} for d < P.  Same
// recurrence as basis_bwd; the level-d adjoints join before level d is swept.
template <int P>
__device__ __forceinline__ void basis_bwd_levels(const Tri<P>& t, const float* gTop, const float (*gLow)[P],
                                                 float* du, float* dU) {
  float g[P + 1];
#pragma unroll
  for (int r = 0; r <= P; ++r) g[r] = gTop[r];
#pragma unroll
  for (int j = P; j >= 1; --j) {
    float gp[P];
#pragma unroll
    for (int r = 0; r < j; ++r) {
      const float x = t.lev[j - 1][r];
      const float D = t.right[r + 1] + t.left[j - r];
      const float inv = 1.f / D;
      const float al = t.left[j - r] * inv;
      const float be = t.right[r + 1] * inv;
      gp[r] = be * g[r] + al * g[r + 1];
      const float dal = x * (g[r + 1] - g[r]);
      *du += dal * inv;
      dU[r + P - j] += dal * (al - 1.f) * inv;
      dU[r + P] -= dal * al * inv;
    }
#pragma unroll
    for (int r = 0; r < j; ++r) g[r] = gp[r] + gLow[j - 1][r];
  }
}

// Reverse of a curve point and of its tangent at one evaluated point: given
// gC = dL/dC (x, y, s) and gD = dL/dC'_xy, with C' = (S' - C_xy W') / W (Eq. 2)
// and the basis derivatives dN from level P-1 of the triangle, adds
// dL/d{x, y, s, w} of the span's control points to dcp, dL/dU of its 2P knots
// to dkn and returns dL/du in *du (0 without KNOTS).
template <int P, bool KNOTS>
__device__ __forceinline__ void curve_tangent_adjoint(const Eval<P>& e, const float* dN, const float gC[3],
                                                      const float gD[2], float dcp[P + 1][4], float dkn[2 * P],
                                                      float* du) {
  const float iw = 1.f / e.W;
  float dSx = 0.f, dSy = 0.f, dW = 0.f;
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    const float nw = dN[l] * e.cp[l].w;
    dSx = fmaf(nw, e.cp[l].x, dSx);
    dSy = fmaf(nw, e.cp[l].y, dSy);
    dW += nw;
  }
  const float Dx = (dSx - e.C[0] * dW) * iw, Dy = (dSy - e.C[1] * dW) * iw;
  // C' = (S' - C W') / W
  const float gSp0 = gD[0] * iw, gSp1 = gD[1] * iw;
  const float gWp = -(gD[0] * e.C[0] + gD[1] * e.C[1]) * iw;
  const float gc0 = gC[0] - gD[0] * dW * iw, gc1 = gC[1] - gD[1] * dW * iw, gc2 = gC[2];
  // C = S / W
  const float gS0 = gc0 * iw, gS1 = gc1 * iw, gS2 = gc2 * iw;
  const float gW = -(gc0 * e.C[0] + gc1 * e.C[1] + gc2 * e.C[2]) * iw - (gD[0] * Dx + gD[1] * Dy) * iw;
  float gN[P + 1], gNp[P + 1];
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    const float4 q = e.cp[l];
    const float N = e.t.N[l], Np = dN[l];
    const float g_nw = gS0 * q.x + gS1 * q.y + gS2 * q.z + gW;    // d/d(N w)
    const float g_npw = gSp0 * q.x + gSp1 * q.y + gWp;             // d/d(N' w)
    dcp[l][0] += q.w * (N * gS0 + Np * gSp0);
    dcp[l][1] += q.w * (N * gS1 + Np * gSp1);
    dcp[l][2] += q.w * N * gS2;
    dcp[l][3] += g_nw * N + g_npw * Np;
    gN[l] = g_nw * q.w;
    gNp[l] = g_npw * q.w;
  }
  float d = 0.f;
  if constexpr (KNOTS) {
    // N'_r = P (tmp[r-1] - tmp[r]), tmp[r] = lev[P-1][r] / D_r, D_r = U[i+r+1] - U[i+r+1-P]
    float gLow[P][P];
#pragma unroll
    for (int a = 0; a < P; ++a)
#pragma unroll
      for (int b = 0; b < P; ++b) gLow[a][b] = 0.f;
#pragma unroll
    for (int r = 0; r < P; ++r) {
      const float D = e.t.right[r + 1] + e.t.left[P - r];
      const float tmp = e.t.lev[P - 1][r] / D;
      const float gt = float(P) * (gNp[r + 1] - gNp[r]);
      gLow[P - 1][r] += gt / D;
      const float gDr = -gt * tmp / D;
      dkn[r + P] += gDr;
      dkn[r] -= gDr;
    }
    basis_bwd_levels<P>(e.t, gN, gLow, &d, dkn);
  }
  *du = d;
}

// Taylor (power-basis) form of the homogeneous curve S_h = sum_l N_l w_l (x_l,
// y_l, 1) on one knot span, about the span's midpoint m:
// S_h(u) = sum_k A[k] (u - m)^k with A[k] = S_h^(k)(m) / k!.  The k-th derivative
// is the degree p-k B-spline of the derivative control points
//   Q^(k)_l = (p-k+1)/(U_{l+p-k+1} - U_l) (Q^(k-1)_l - Q^(k-1)_{l-1})
// over the level p-k functions of the span triangle at m.
template <int P>
struct SpanPoly {
  float m;
  float A[P + 1][3];
};

template <int P>
__device__ __forceinline__ void span_poly(const float4* key, const CurveRef& cr, const float* U, int i,
                                          SpanPoly<P>& sp) {
  const float m = 0.5f * (U[i] + U[i + 1]);
  Tri<P> t;
  basis_fwd<P>(U, i, m, t);
  float Q[P + 1][3];
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    const float4 q = key[cr.key0 + cp_to_key(i - P + l, P, cr.closed, cr.nk)];
    Q[l][0] = q.w * q.x;
    Q[l][1] = q.w * q.y;
    Q[l][2] = q.w;
  }
  sp.m = m;
  float fact = 1.f;
#pragma unroll
  for (int k = 0; k <= P; ++k) {
    if (k > 0) {
      fact *= float(k);
      // Q^(k) from Q^(k-1), highest l first so that Q[l - 1] still holds level k-1
#pragma unroll
      for (int l = P; l >= k; --l) {
        const float c = float(P - k + 1) / (U[i + l - k + 1] - U[i - P + l]);
#pragma unroll
        for (int e = 0; e < 3; ++e) Q[l][e] = c * (Q[l][e] - Q[l - 1][e]);
      }
    }
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
    for (int l = k; l <= P; ++l) {
      const float n = (k == 0) ? t.N[l] : t.lev[P - k < P ? P - k : 0][l - k];
      a0 = fmaf(n, Q[l][0], a0);
      a1 = fmaf(n, Q[l][1], a1);
      a2 = fmaf(n, Q[l][2], a2);
    }
    const float inv = 1.f / fact;
    sp.A[k][0] = a0 * inv;
    sp.A[k][1] = a1 * inv;
    sp.A[k][2] = a2 * inv;
  }
}

// Sum of 8 values over the 32 lanes of a warp in 9 shuffles: each exchange
// step hands half of the remaining values to the partner lane.  On return the
// lanes with (lane & 3) == 0 hold the totals, value (lane >> 2) in lane.
__device__ __forceinline__ float warp_sum8(const float v[8]) {
  const int lane = threadIdx.x & 31;
  float b[4], c[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float send = h16 ? v[i] : v[i + 4];
    const float keep = h16 ? v[i + 4] : v[i];
    b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = h8 ? b[i] : b[i + 2];
    const float keep = h8 ? b[i + 2] : b[i];
    c[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float d = (h4 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h4 ? c[0] : c[1], 4);
  d += __shfl_xor_sync(0xffffffffu, d, 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  return d;
}

// Sum of 4 values over the 32 lanes in 6 shuffles (the same exchange scheme):
// on return value k of the total sits in the lanes with (lane >> 3) == k.
__device__ __forceinline__ float warp_sum4(const float v[4]) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  float b[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float send = h16 ? v[i] : v[i + 2];
    const float keep = h16 ? v[i + 2] : v[i];
    b[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float d = (h8 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h8 ? b[0] : b[1], 8);
  d += __shfl_xor_sync(0xffffffffu, d, 4);
  d += __shfl_xor_sync(0xffffffffu, d, 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  return d;
}

// K exclusive scans over the same items in one sweep of a single block:
// get(i, v) gives item i's K values, put(i, off) receives their K offsets,
// tot the K totals.  Each thread takes a run of up to kScanRun consecutive
// items per pass (all its reads in flight together), the block scans the
// runs' sums, and each thread hands out its items' offsets.
constexpr int kScanRun = 4;

template <int K, class Get, class Put>
__device__ void block_scan_multi(int n, Get get, Put put, long long tot[K]) {
  __shared__ long long s_carry[K];
  __shared__ long long s_warp[K][32];
  if (threadIdx.x < K) s_carry[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nb = blockDim.x;
  for (int base = 0; base < n; base += nb * kScanRun) {
    const int run = min(kScanRun, (n - base + nb - 1) / nb);   // items per thread in this pass
    const int i0 = base + threadIdx.x * run;
    long long v[kScanRun][K], x[K];
#pragma unroll
    for (int j = 0; j < kScanRun; ++j) {
#pragma unroll
      for (int k = 0; k < K; ++k) v[j][k] = 0;
      if (j < run && i0 + j < n) get(i0 + j, v[j]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      x[k] = 0;
#pragma unroll
      for (int j = 0; j < kScanRun; ++j) x[k] += v[j][k];
    }
    long long sum[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      sum[k] = x[k];
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x[k], o);
        if (lane >= o) x[k] += y;
      }
      if (lane == 31) s_warp[k][w] = x[k];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        long long t = lane < nw ? s_warp[k][lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
          const long long y = __shfl_up_sync(0xffffffffu, t, o);
          if (lane >= o) t += y;
        }
        if (lane < nw) s_warp[k][lane] = t;
      }
    }
    __syncthreads();
    long long off[K];
#pragma unroll
    for (int k = 0; k < K; ++k) off[k] = s_carry[k] + (w > 0 ? s_warp[k][w - 1] : 0) + x[k] - sum[k];
#pragma unroll
    for (int j = 0; j < kScanRun; ++j) {
      if (j < run && i0 + j < n) put(i0 + j, off);
#pragma unroll
      for (int k = 0; k < K; ++k) off[k] += v[j][k];
    }
    __syncthreads();
    if (threadIdx.x == nb - 1)
#pragma unroll
      for (int k = 0; k < K; ++k) s_carry[k] = off[k];
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < K; ++k) tot[k] = s_carry[k];
}

// Runtime degree -> template dispatch.
#define NS_DISPATCH_P(p, ...)                     \
  switch (p) {                                    \
    case 1: { constexpr int P = 1; __VA_ARGS__; } break; \
    case 2: { constexpr int P = 2; __VA_ARGS__; } break; \
    case 3: { constexpr int P = 3; __VA_ARGS__; } break; \
    case 4: { constexpr int P = 4; __VA_ARGS__; } break; \
    case 5: { constexpr int P = 5; __VA_ARGS__; } break; \
    default: break;                               \
  }

// Parameter of sample l of a contour curve (open: [first x kappa, M samples,
// last x kappa]; closed: M samples without repeating the start).
__device__ __forceinline__ float contour_u(const CurvePlan& pl, int l, int kappa) {
  float t;
  if (pl.kind == kOpen) {
    const int j = l - kappa;
    t = j <= 0 ? 0.f : (j >= pl.M - 1 ? 1.f : float(j) / float(pl.M - 1));
  } else {
    t = float(l) / float(pl.M);
  }
  return pl.a + t * (pl.b - pl.a);
}

__device__ __forceinline__ float contour_t(const CurvePlan& pl, int l, int kappa) {
  if (pl.kind == kOpen) {
    const int j = l - kappa;
    return j <= 0 ? 0.f : (j >= pl.M - 1 ? 1.f : float(j) / float(pl.M - 1));
  }
  return float(l) / float(pl.M);
}

// Task -> curve from the table nurbs_sample writes (fill tasks first, then the
// contour tasks); tasks beyond the table (only when the Gaussian capacity
// overflowed) fall back to the search below.
__device__ __forceinline__ int curve_of_task(const CurvePlan* __restrict__ plan, const int* __restrict__ order,
                                             int nc, int task, bool fill);
__device__ __forceinline__ int task_curve(const int* __restrict__ tmap, long long tcap, int n_fill,
                                          const CurvePlan* __restrict__ plan, const int* __restrict__ order, int nc,
                                          int task, bool fill) {
  const long long t = fill ? task : (long long)n_fill + task;
  return t < tcap ? tmap[t] : curve_of_task(plan, order, nc, task, fill);
}

// Fill tasks of a curve's nx x ny grid: its T x T tiles, row-major.
__host__ __device__ __forceinline__ int fill_task_count(int nx, int ny, int T) {
  return ((nx + T - 1) / T) * ((ny + T - 1) / T);
}

// Grid point (ix, iy) of thread t (0..T^2-1) in fill task k (T x T tiles) of a
// curve with an nx x ny grid; false past the grid.
__device__ __forceinline__ bool fill_task_point(int k, int nx, int ny, int t, int T, int& ix, int& iy) {
  const int tcols = (nx + T - 1) / T;
  ix = (k % tcols) * T + (t % T);
  iy = (k / tcols) * T + (t / T);
  return ix < nx && iy < ny;
}

// The fill tile edge of a sampling setting (0 -> 16).
__host__ __device__ __forceinline__ int fill_tile_of(int v) { return v == 8 ? 8 : 16; }

// Task -> curve map.  Contour tasks are 256 samples of one curve, fill tasks
// 16 x 16 tiles of one curve's grid; fill tasks and
// contour tasks are numbered separately, each kind in front-to-back curve
// order, and a curve's chunk_off counts the tasks of its own kind before it.
// Curves of the other kind contribute no tasks to the count, so over the
// ordered list the offsets of one kind never decrease, and the largest position
// whose offset is <= task is the curve that owns it.
__device__ __forceinline__ int curve_of_task(const CurvePlan* __restrict__ plan, const int* __restrict__ order,
                                             int nc, int task, bool fill) {
  int lo = 0, hi = nc - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const CurvePlan& q = plan[order[mid]];
    const int off = (q.kind == kFill) == fill ? q.chunk_off : q.pad[0];
    if (off <= task) lo = mid; else hi = mid - 1;
  }
  return order[lo];
}

}  // namespace ns
