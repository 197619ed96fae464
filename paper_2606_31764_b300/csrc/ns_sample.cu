// nurbs_sample: curves -> Gaussians (paper §3.1-§3.3).
//
// Kernels, in launch order:
//   k_plan_forms    one block per curve: validation, scene order, knot vector
//                   (exact running sum stored as FP32 high and low parts);
//                   then one thread per span: the span's Taylor form of the
//                   rational curve (Eq. 1), and reciprocals of knot
//                   differences for filled curves
//   k_plan_length   one block per curve: arc length by N_L-node midpoint
//                   quadrature of |C'| (Eq. 2-3, block reduction), counts
//   k_scan_boundary one block: boundary-point offsets of filled curves
//   k_boundary      one thread per boundary point b_i of the filled curves,
//                   evaluated in double-float arithmetic
//   k_boundary_box  one warp per filled curve: the polyline's padded and
//                   clipped box, the fill grid origin (high and low parts) and
//                   size, the points made relative to the origin, and the
//                   bounding box of each cluster of 8 segments (the lower
//                   bounds the fill SDF's segment lists test)
//   k_scan_gauss    one block: Gaussian and task offsets in front-to-back order
//   k_fill_sdf      persistent over the fill tasks (16 x 16 tiles of a curve's
//                   grid): the SDF of Eq. S1-S3 from the band of segments
//                   near the tile and per-row crossing lists, the fill
//                   opacity of Eq. 7 and the records (Eq. 6)
//   k_emit          persistent over the contour tasks: 256 samples of a
//                   stroke per block iteration (Eq. 4-5)
#include <cuda_runtime.h>
#include <float.h>

#include <algorithm>

#include "ns_internal.cuh"

namespace ns {

// Boundary points are evaluated in double-float arithmetic: every value is an
// unevaluated sum hi + lo of two floats (about 48 significant bits), built
// from the error-free transformations TwoSum (Knuth) and TwoProduct (Dekker;
// here with the fused multiply-add, as Ogita, Rump and Oishi write it).  The
// knot vector (the same sums as k_plan_forms), the parameters, the Cox-de Boor
// triangle and the rational quotient of Eq. 1 all carry that precision.
// FP32 evaluation at pixel coordinates near 1000 has errors of about 1e-4 px,
// which the grid origin and, through the sigmoid of Eq. 7, the fill opacities
// inherit; FP64 gives the same precision as double-float but runs far slower
// on this part.
struct df {
  float h, l;
};
__device__ __forceinline__ df df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = df_two_sum(x.h, y.h);
  const df t = df_two_sum(x.l, y.l);
  s = df_fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return df_fast_two_sum(s.h, __fadd_rn(s.l, t.l));
}
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df{-y.h, -y.l}); }
__device__ __forceinline__ df df_mul(df x, df y) {
  const float p = __fmul_rn(x.h, y.h);
  const float e = __fmaf_rn(x.h, y.h, -p);   // exact error of the product
  return df_fast_two_sum(p, __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, e)));
}
__device__ __forceinline__ df df_mulf(df x, float y) {
  const float p = __fmul_rn(x.h, y);
  return df_fast_two_sum(p, __fmaf_rn(x.l, y, __fmaf_rn(x.h, y, -p)));
}
// 1/d: the float reciprocal q refined by one Newton step, q + q (1 - d q),
// with the residual 1 - d q formed exactly enough in double-float.
__device__ __forceinline__ df df_rcp(df d) {
  const float q = 1.f / d.h;
  const df r = df_sub(df{1.f, 0.f}, df_mulf(d, q));
  return df_fast_two_sum(q, __fmul_rn(q, r.h));
}
__device__ __forceinline__ bool df_less(df a, df b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ double df_to_double(df a) { return double(a.h) + double(a.l); }

constexpr int kPlanThreads = 128;
constexpr int kCluster = 8;       // consecutive segments per bounding-box cluster

__device__ __forceinline__ float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float s = 0.f;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  return red[0];
}

// |C'_xy(u)| (Eq. 2) from the span's Taylor form: C = S/W, C' = (S' - C W')/W.
template <int P>
__device__ __forceinline__ float span_speed(const SpanPoly<P>& sp, float u) {
  const float t = u - sp.m;
  float S0 = sp.A[P][0], S1 = sp.A[P][1], W = sp.A[P][2];
  float D0 = 0.f, D1 = 0.f, DW = 0.f;
#pragma unroll
  for (int k = P - 1; k >= 0; --k) {
    D0 = fmaf(D0, t, S0);
    D1 = fmaf(D1, t, S1);
    DW = fmaf(DW, t, W);
    S0 = fmaf(S0, t, sp.A[k][0]);
    S1 = fmaf(S1, t, sp.A[k][1]);
    W = fmaf(W, t, sp.A[k][2]);
  }
  // the reciprocal and the square root of the special-function unit (about
  // 1e-7 relative each; the sum over the nodes carries more rounding than that)
  const float iw = __fdividef(1.f, W);
  const float dx = (D0 - S0 * iw * DW) * iw, dy = (D1 - S1 * iw * DW) * iw;
  const float v2 = dx * dx + dy * dy;
  return v2 > 0.f ? v2 * rsqrtf(v2) : 0.f;
}

// The Taylor form {m, A[0..P][3]} of every non-empty span of every curve, one
// row of kFormStride floats per knot slot (the row of the knot that starts
// the span), written by k_plan_forms and read by the arc-length nodes.
static_assert(kFormStride >= 1 + 3 * (kMaxP + 1), "a span form row holds m and A[0..p][3]");

template <int P>
__device__ __forceinline__ void load_form(const float* __restrict__ d, SpanPoly<P>& sp) {
  sp.m = d[0];
#pragma unroll
  for (int k = 0; k <= P; ++k) {
    sp.A[k][0] = d[1 + 3 * k];
    sp.A[k][1] = d[2 + 3 * k];
    sp.A[k][2] = d[3 + 3 * k];
  }
}

// Each thread sums a contiguous run of the N_L midpoint nodes (Eq. 3),
// loading a span's form whenever its run enters that span.
template <int P>
__device__ float arc_length_part(const float* __restrict__ forms, const CurveRef& cr, const float* __restrict__ U,
                                 float a, float b, int NL) {
  const float du = (b - a) / float(NL);
  const int per = (NL + blockDim.x - 1) / blockDim.x;
  const int j0 = threadIdx.x * per, j1 = min(NL, j0 + per);
  const float* F = forms + (long long)cr.knot0 * kFormStride;   // knot0 = 0 when forms is the curve's own
  float acc = 0.f;
  SpanPoly<P> sp;
  int span = -1;
  float hi = 0.f;
  for (int j = j0; j < j1; ++j) {
    const float u = a + (float(j) + 0.5f) * du;
    if (span < 0 || !(u < hi)) {
      span = find_span(U, P, cr.n, u);
      hi = span < cr.n ? U[span + 1] : 3.0e38f;
      load_form<P>(F + (long long)span * kFormStride, sp);
    }
    acc += span_speed<P>(sp, u);
  }
  return acc * du;
}

// k_plan_forms: one block per curve.  Thread 0 validates the curve, places it
// in its scene's front-to-back order and builds the knot vector (§3.1: open
// -> p zero intervals on both sides; closed -> the last p core intervals
// before, the first p after; cumulative sum from 0) as an exact running sum
// kept as FP32 high and low parts.  Then, one thread per span, the Taylor
// form of the rational curve on each non-empty span (span_poly), and for
// filled curves the reciprocals of the knot differences of widths 1..p
// (k_boundary).
constexpr int kFormThreads = 64;
constexpr int kTauStage = 1024;   // intervals staged (longer curves read them from global memory)

template <int P>
__device__ void span_forms(const float4* key, const CurveRef& cr, const float* U, float* F) {
  const int nspan = cr.n - P + 1;
  for (int sidx = threadIdx.x; sidx < nspan; sidx += blockDim.x) {
    const int i = P + sidx;
    if (!(U[i] < U[i + 1])) continue;   // empty span: never the span of a node
    SpanPoly<P> sp;
    span_poly<P>(key, cr, U, i, sp);
    float* d = F + (long long)i * kFormStride;
    d[0] = sp.m;
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      d[1 + 3 * k] = sp.A[k][0];
      d[2 + 3 * k] = sp.A[k][1];
      d[3 + 3 * k] = sp.A[k][2];
    }
  }
}

__global__ void __launch_bounds__(kFormThreads) k_plan_forms(ns_curves cv, CurvePlan* plan, float* knots,
                                                             float* knots_lo, float2* krcp, int* order,
                                                             DevState* st, float* forms) {
  grid_dep_wait();
  __shared__ float s_tau[kTauStage];
  __shared__ int s_ok;
  const int c = blockIdx.x;
  const CurveRef cr = curve_ref(cv, c);
  float* U = knots + cr.knot0;
  float* Ulo = knots_lo + cr.knot0;
  const int t0 = cv.tau_offset[c];
  const bool tau_staged = cr.ntau >= 0 && cr.ntau <= kTauStage && t0 >= 0 && cv.tau_offset[c + 1] <= cv.n_taus;
  if (tau_staged)
    for (int q = threadIdx.x; q < cr.ntau; q += blockDim.x) s_tau[q] = cv.tau[t0 + q];
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = cr.p >= 1 && cr.p <= kMaxP && cr.key0 >= 0 && cr.nk >= 0 && t0 >= 0 && cr.ntau >= 0 &&
             cv.key_offset[c + 1] <= cv.n_keys && cv.tau_offset[c + 1] <= cv.n_taus;
    if (ok) ok = cr.closed ? (cr.nk >= cr.p && cr.nk >= 2 && cr.ntau == cr.nk)
                           : (cr.nk >= cr.p + 1 && cr.ntau == cr.nk - cr.p);
    if (ok && cr.filled && !cr.closed) ok = 0;
    // a stroke of a degree the caller's launch hint leaves out
    if (ok && (cv.stroke_degrees & 1) && !cr.filled && !(cv.stroke_degrees & (1 << cr.p))) ok = 0;
    // scene and front-to-back position: reverse order inside the scene
    int s = 0, s0 = 0, s1 = cv.n_curves;
    if (cv.scene_curve_offset) {
      int lo = 0, hi = cv.n_scenes - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cv.scene_curve_offset[mid] <= c) lo = mid; else hi = mid - 1;
      }
      s = lo;
      s0 = cv.scene_curve_offset[s];
      s1 = cv.scene_curve_offset[s + 1];
    }
    if (s0 <= c && c < s1 && s1 <= cv.n_curves) order[s0 + (s1 - 1 - c)] = c;
    else ok = 0;   // inconsistent scene offsets
    plan[c].scene = s;
    if (ok) {
      const float* tau = tau_staged ? s_tau : cv.tau + t0;
      const int p = cr.p, nt = cr.ntau;
      const int n_int = nt + 2 * p;
      // exact running sum as hi + lo: TwoSum keeps each addition's rounding
      // error, which the low part collects (the sums of float intervals need
      // far fewer than 48 bits)
      float acc_h = 0.f, acc_l = 0.f, u_p = 0.f, u_end = 0.f;
      U[0] = 0.f;
      Ulo[0] = 0.f;
      // the interval of step q: open curves pad with zeros, closed curves
      // wrap (from interval nt - p on, modulo nt)
      int k = cr.closed ? ((nt - p) % nt + nt) % nt : 0;
      for (int q = 0; q < n_int; ++q) {
        float v;
        if (!cr.closed) {
          v = (q < p || q >= p + nt) ? 0.f : tau[q - p];
        } else {
          v = tau[k];
          if (++k == nt) k = 0;
        }
        if (!(v >= 0.f)) ok = 0;   // negative or NaN interval
        const df t = df_two_sum(acc_h, v);
        acc_h = t.h;
        acc_l = __fadd_rn(acc_l, t.l);
        const df u = df_fast_two_sum(acc_h, acc_l);
        U[q + 1] = u.h;
        Ulo[q + 1] = u.l;
        if (q + 1 == p) u_p = u.h;
        if (q + 1 == cr.n + 1) u_end = u.h;
      }
      if (ok && !(u_end > u_p)) ok = 0;   // empty domain
    }
    if (!ok) {
      atomicCAS(&st->bad_curve, -1, c);
      raise_status(st, NS_ERR_INVALID_CURVE);
      plan[c].kind = kNone;
      plan[c].count = 0;
      plan[c].M = 0;
      plan[c].L = 0.f;
    } else {
      plan[c].kind = cr.filled ? kFill : (cr.closed ? kClosedStroke : kOpen);
    }
    s_ok = ok;
  }
  __syncthreads();   // thread 0's knots are visible to the block
  if (!s_ok) return;
  const float4* key = reinterpret_cast<const float4*>(cv.key);
  NS_DISPATCH_P(cr.p, span_forms<P>(key, cr, U, forms + (long long)cr.knot0 * kFormStride));
  if (cr.filled) {
    // reciprocals of the knot differences of width 1..p (double-float), for
    // the boundary points' Cox-de Boor triangle
    const int nkn = cr.ntau + 2 * cr.p + 1;
    float2* rc = krcp + (long long)kMaxP * cr.knot0;
    for (int q = threadIdx.x; q < cr.p * nkn; q += blockDim.x) {
      const int j = q / nkn + 1, kk = q - (j - 1) * nkn;
      const df d = kk + j < nkn ? df_sub(df{U[kk + j], Ulo[kk + j]}, df{U[kk], Ulo[kk]}) : df{0.f, 0.f};
      const df r = d.h > 0.f ? df_rcp(d) : df{0.f, 0.f};
      rc[(j - 1) * nkn + kk] = make_float2(r.h, r.l);
    }
  }
}

// k_plan_length: one block per valid curve: the arc length by the N_L-node
// midpoint rule of Eq. 3 on the span forms (block reduction), then the
// counts (§3.2, §3.3).  The curve's knots and forms are staged in shared
// memory when they fit.
constexpr int kLenStage = 128;   // knots (and span rows) staged per curve

__global__ void __launch_bounds__(kPlanThreads, 8) k_plan_length(ns_curves cv, ns_sample_params sp, CurvePlan* plan,
                                                                 const float* __restrict__ knots,
                                                                 const float* __restrict__ forms) {
  grid_dep_wait();
  __shared__ float red[32];
  __shared__ float sU[kLenStage];
  __shared__ float sF[kLenStage * kFormStride];
  const int c = blockIdx.x;
  const int kind = plan[c].kind;
  if (kind == kNone) return;
  CurveRef cr = curve_ref(cv, c);
  const float* U = knots + cr.knot0;
  const float* F = forms + (long long)cr.knot0 * kFormStride;
  const int nkn = cr.ntau + 2 * cr.p + 1;
  if (nkn <= kLenStage) {   // spans p..n < nkn
    for (int q = threadIdx.x; q < nkn; q += blockDim.x) sU[q] = U[q];
    // the rows of spans p..n (the others are never read)
    const int f0 = cr.p * kFormStride, f1 = (cr.n + 1) * kFormStride;
    for (int q = f0 + threadIdx.x; q < f1; q += blockDim.x) sF[q] = F[q];
    __syncthreads();
    U = sU;
    F = sF;
  }
  const float a = U[cr.p], b = U[cr.n + 1];
  const int NL = sp.nl_mult * max(cv.width, cv.height);
  float part = 0.f;
  cr.knot0 = 0;   // F is the curve's own table
  NS_DISPATCH_P(cr.p, part = arc_length_part<P>(F, cr, U, a, b, NL));
  const float L = block_sum(part, red);
  if (threadIdx.x == 0) {
    CurvePlan pl;
    pl.L = L;
    pl.a = a;
    pl.b = b;
    pl.x0 = pl.y0 = 0.f;
    pl.nx = pl.ny = 0;
    pl.h = 0.f;
    pl.kind = kind;
    if (kind == kFill) {
      pl.M = max(3, int(ceilf(sp.delta_b * L)));
      pl.count = 0;   // set by k_boundary_box
    } else if (kind == kClosedStroke) {
      pl.M = max(1, int(ceilf(sp.delta_c * L)));
      pl.count = pl.M;
    } else {
      pl.M = max(2, int(ceilf(sp.delta_c * L)));
      pl.count = pl.M + 2 * sp.kappa;
    }
    pl.scene = plan[c].scene;
    pl.g_off = pl.b_off = pl.chunk_off = 0;
    pl.pad[0] = 0;
    plan[c] = pl;
  }
}

__global__ void k_scan_boundary(int nc, CurvePlan* plan, DevState* st, long long bcap, int* boffs) {
  grid_dep_wait();
  // the offsets also go to a packed array, which k_boundary searches
  long long t1[1];
  block_scan_multi<1>(
      nc, [&](int c, long long v[1]) { v[0] = plan[c].kind == kFill ? plan[c].M : 0; },
      [&](int c, const long long off[1]) {
        plan[c].b_off = int(off[0]);
        boffs[c] = int(off[0]);
      },
      t1);
  const long long tot = t1[0];
  if (threadIdx.x == 0) {
    st->b_total = (unsigned long long)tot;
    st->b_count = int(tot < bcap ? tot : bcap);
    if (tot > bcap) raise_status(st, NS_ERR_CAPACITY);
  }
}

// C_xy(u) on span i in double-float, the knots U given as high and low parts.
template <int P>
__device__ __forceinline__ void curve_xy_df(const float4* __restrict__ key, const CurveRef& cr,
                                            const float* __restrict__ Uh, const float* __restrict__ Ul,
                                            const float2* __restrict__ rc, int ld, int i, df u, df& x, df& y) {
  df N[P + 1], left[P + 1], right[P + 1];
  N[0] = df{1.f, 0.f};
#pragma unroll
  for (int j = 1; j <= P; ++j) {
    left[j] = df_sub(u, df{Uh[i + 1 - j], Ul[i + 1 - j]});
    right[j] = df_sub(df{Uh[i + j], Ul[i + j]}, u);
    df saved = df{0.f, 0.f};
#pragma unroll
    for (int r = 0; r < j; ++r) {
      // 1 / (U[i+r+1] - U[i+1-j+r]), positive on a non-empty span
      const float2 inv = rc[(j - 1) * ld + i + 1 - j + r];
      const df temp = df_mul(N[r], df{inv.x, inv.y});
      N[r] = df_add(saved, df_mul(right[r + 1], temp));
      saved = df_mul(left[j - r], temp);
    }
    N[j] = saved;
  }
  df Sx{0.f, 0.f}, Sy{0.f, 0.f}, W{0.f, 0.f};
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    const float4 q = key[cr.key0 + cp_to_key(i - P + l, P, cr.closed, cr.nk)];
    const df nw = df_mulf(N[l], q.w);
    Sx = df_add(Sx, df_mulf(nw, q.x));
    Sy = df_add(Sy, df_mulf(nw, q.y));
    W = df_add(W, nw);
  }
  const df iw = df_rcp(W);
  x = df_mul(Sx, iw);
  y = df_mul(Sy, iw);
}

// One thread per boundary point of every filled curve: b_j = C_xy(a + (j/B)
// (b - a)), j < B (closed rule), evaluated in double-float; writes the
// absolute FP32 copy, the curve table and, in the local array, the
// double-float pair {x.h, y.h, x.l, y.l} (k_boundary_box makes it relative to
// the grid origin).  The span is searched on the FP32 knots and settled on
// the double-float ones.
__global__ void __launch_bounds__(256) k_boundary(ns_curves cv, const CurvePlan* __restrict__ plan,
                                                  const float* __restrict__ knots, const float* __restrict__ knots_lo,
                                                  const float2* __restrict__ krcp,
                                                  const DevState* __restrict__ st, float2* bpts, int* bcurve,
                                                  float4* bloc, long long bcap, const int* __restrict__ boffs) {
  grid_dep_wait();
  const long long nb = min((long long)st->b_count, bcap);
  const int nc = cv.n_curves;
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < nb;
       o += (long long)gridDim.x * blockDim.x) {
    // the curve: the largest c with b_off <= o (curves without points share
    // the offset of the next one, and the largest index is the filled curve);
    // searched in the packed offsets, whose last levels share cache lines
    int lo = 0, hi = nc - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (boffs[mid] <= o) lo = mid; else hi = mid - 1;
    }
    const int c = lo;
    const CurvePlan pl = plan[c];
    const int j = int(o - pl.b_off);
    if (pl.kind != kFill || j < 0 || j >= pl.M) continue;
    const CurveRef cr = curve_ref(cv, c);
    const float* Uh = knots + cr.knot0;
    const float* Ul = knots_lo + cr.knot0;
    const df a{Uh[cr.p], Ul[cr.p]}, b{Uh[cr.n + 1], Ul[cr.n + 1]};
    // t = j / B as a double-float: the float quotient plus the exact remainder over B
    const float B = float(pl.M);
    const float q = float(j) / B;
    const df t = df_fast_two_sum(q, __fmaf_rn(-q, B, float(j)) / B);
    const df u = df_add(a, df_mul(t, df_sub(b, a)));
    const int p = cr.p;
    int i = find_span(Uh, p, cr.n, u.h);
    while (i < cr.n && !df_less(u, df{Uh[i + 1], Ul[i + 1]})) ++i;
    while (i > p && df_less(u, df{Uh[i], Ul[i]})) --i;
    while (i > p && !df_less(df{Uh[i], Ul[i]}, df{Uh[i + 1], Ul[i + 1]})) --i;
    df x{0.f, 0.f}, y{0.f, 0.f};
    NS_DISPATCH_P(p, curve_xy_df<P>(reinterpret_cast<const float4*>(cv.key), cr, Uh, Ul,
                                    krcp + (long long)kMaxP * cr.knot0, cr.ntau + 2 * p + 1, i, u, x, y));
    bpts[o] = make_float2(x.h, y.h);
    bloc[o] = make_float4(x.h, y.h, x.l, y.l);
    bcurve[o] = c;
  }
}

// One warp per filled curve: the box of its boundary points (double-float
// comparisons), the grid origin and size decided in double precision (a
// handful of scalar operations), the origin stored as a high part (plan) and
// a low part (glo), and the points rewritten relative to it as high and low
// floats (bloc) -- what the signed distance of Eq. S1-S3, the fill chain and
// the fill-layer blend work with.
__global__ void __launch_bounds__(256) k_boundary_box(ns_curves cv, ns_sample_params sp, CurvePlan* plan,
                                                      const float* __restrict__ knots, float4* bloc, float2* glo,
                                                      long long bcap, int4* lbox, DevState* st, float4* cbox) {
  grid_dep_wait();
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c == 0 && lane == 0) {
    st->cull_thr = sp.fill_cull;   // the threshold k_fill_sdf counts for
    st->sdf_next = 0;
  }
  if (c < cv.n_curves && lane == 0) lbox[c] = make_int4(0x7fffffff, 0x7fffffff, -1, -1);
  if (c >= cv.n_curves) return;
  const CurvePlan pl = plan[c];
  if (pl.kind != kFill) return;
  const bool whole = (long long)pl.b_off + pl.M <= bcap;   // else the polyline overflowed: box from what exists
  const int M = whole ? pl.M : int(max(0LL, min((long long)pl.M, bcap - pl.b_off)));
  df box[4] = {df{FLT_MAX, 0.f}, df{FLT_MAX, 0.f}, df{-FLT_MAX, 0.f}, df{-FLT_MAX, 0.f}};
  for (int j = lane; j < pl.M; j += 32) {
    df x, y;
    if (j < M) {
      const float4 v = bloc[pl.b_off + j];
      x = df{v.x, v.z};
      y = df{v.y, v.w};
    } else {
      // past the boundary capacity: evaluated in FP32 only to size the grid
      // (NS_ERR_CAPACITY is raised, the curve emits nothing)
      const CurveRef cr = curve_ref(cv, c);
      const float* U = knots + cr.knot0;
      const float u = pl.a + (float(j) / float(pl.M)) * (pl.b - pl.a);
      float2 q = make_float2(0.f, 0.f);
      NS_DISPATCH_P(cr.p, {
        Eval<P> e;
        eval_curve<P>(reinterpret_cast<const float4*>(cv.key), cr, U, find_span(U, P, cr.n, u), u, e);
        q = make_float2(e.C[0], e.C[1]);
      });
      x = df{q.x, 0.f};
      y = df{q.y, 0.f};
    }
    if (df_less(x, box[0])) box[0] = x;
    if (df_less(y, box[1])) box[1] = y;
    if (df_less(box[2], x)) box[2] = x;
    if (df_less(box[3], y)) box[3] = y;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      const df x{__shfl_xor_sync(0xffffffffu, box[k].h, o), __shfl_xor_sync(0xffffffffu, box[k].l, o)};
      if (k < 2 ? df_less(x, box[k]) : df_less(box[k], x)) box[k] = x;
    }
  }
  const double xmin = df_to_double(box[0]), ymin = df_to_double(box[1]);
  const double xmax = df_to_double(box[2]), ymax = df_to_double(box[3]);
  const double padx = double(sp.pad_frac) * (xmax - xmin);
  const double pady = double(sp.pad_frac) * (ymax - ymin);
  const double x0 = fmax(0.0, xmin - padx), x1 = fmin(double(cv.width), xmax + padx);
  const double y0 = fmax(0.0, ymin - pady), y1 = fmin(double(cv.height), ymax + pady);
  const float x0h = float(x0), y0h = float(y0);
  const df ox{x0h, float(x0 - double(x0h))}, oy{y0h, float(y0 - double(y0h))};
  __syncwarp();
  for (int j = lane; j < M; j += 32) {
    const float4 v = bloc[pl.b_off + j];
    const df lx = df_sub(df{v.x, v.z}, ox), ly = df_sub(df{v.y, v.w}, oy);
    bloc[pl.b_off + j] = make_float4(lx.h, ly.h, lx.l, ly.l);
  }
  if (whole) {
    // the box of each cluster of kCluster segments (grid-local high parts),
    // at the index of the cluster's first point; the warp's own points above
    // are visible to its lanes after the warp barrier
    __syncwarp();
    const int B = pl.M;
    for (int k = lane * kCluster; k < B; k += 32 * kCluster) {
      float cx0 = FLT_MAX, cx1 = -FLT_MAX, cy0 = FLT_MAX, cy1 = -FLT_MAX;
      for (int j = k; j < min(B, k + kCluster); ++j) {
        const float4 b0 = bloc[pl.b_off + j];
        const float4 b1 = bloc[pl.b_off + (j + 1 == B ? 0 : j + 1)];
        cx0 = fminf(cx0, fminf(b0.x, b1.x));
        cx1 = fmaxf(cx1, fmaxf(b0.x, b1.x));
        cy0 = fminf(cy0, fminf(b0.y, b1.y));
        cy1 = fmaxf(cy1, fmaxf(b0.y, b1.y));
      }
      cbox[pl.b_off + k] = make_float4(cx0, cx1, cy0, cy1);
    }
  }
  if (lane == 0) {
    const double h = double(sp.h);
    const int nx = x1 > x0 ? int(ceil((x1 - x0) / h)) : 0;
    const int ny = y1 > y0 ? int(ceil((y1 - y0) / h)) : 0;
    plan[c].x0 = x0h;
    plan[c].y0 = y0h;
    glo[c] = make_float2(ox.l, oy.l);
    plan[c].nx = nx;
    plan[c].ny = ny;
    plan[c].h = sp.h;
    plan[c].count = nx * ny;
  }
}

// Gaussian offsets over all curves (front to back), and task offsets per kind:
// chunk_off numbers a curve's tasks among the curves of its kind; pad[0] holds
// the task count of the other kind before it, so that each kind's offsets
// can be searched over the one ordered list (see curve_of_task).
__global__ void k_scan_gauss(int nc, CurvePlan* plan, const int* order, DevState* st, long long gcap,
                             int* g_count_out, int ftile, int* bmix, long long n_bins) {
  grid_dep_wait();
  // the binning blocks (kBinItems Gaussians each) that hold a stroke's
  // Gaussians are marked once the offsets are known; the others hold fill
  // Gaussians only (the binning skips them with fill layers)
  for (long long i = threadIdx.x; i < n_bins; i += blockDim.x) bmix[i] = 0;
  // three scans in front-to-back order: Gaussians, fill tasks, contour tasks;
  // a curve's own tasks start at chunk_off, pad[0] holds the other kind's
  // offset (the search of curve_of_task)
  long long t3[3];
  block_scan_multi<3>(
      nc,
      [&](int f, long long v[3]) {
        const CurvePlan& q = plan[order[f]];
        v[0] = q.count;
        v[1] = q.kind == kFill ? fill_task_count(q.nx, q.ny, ftile) : 0;
        v[2] = q.kind != kFill ? (q.count + kChunk - 1) / kChunk : 0;
      },
      [&](int f, const long long off[3]) {
        CurvePlan& q = plan[order[f]];
        q.g_off = int(off[0] < 0x7fffffff ? off[0] : 0x7fffffff);
        q.chunk_off = int(q.kind == kFill ? off[1] : off[2]);
        q.pad[0] = int(q.kind == kFill ? off[2] : off[1]);
        if (q.kind != kFill && q.count > 0 && off[0] < gcap) {
          const long long e = min(off[0] + q.count, gcap) - 1;
          for (long long b = off[0] / kBinItems; b <= e / kBinItems && b < n_bins; ++b) bmix[b] = 1;
        }
      },
      t3);
  const long long tot = t3[0], ftasks = t3[1], ctasks = t3[2];
  if (threadIdx.x == 0) {
    st->g_total = (unsigned long long)tot;
    const int gc = int(tot < gcap ? tot : gcap);
    st->g_count = gc;
    st->n_chunks = int(ftasks);
    st->n_ctasks = int(ctasks);
    if (g_count_out) *g_count_out = gc;
    if (tot > gcap) raise_status(st, NS_ERR_CAPACITY);
  }
}

// Task -> curve table: one warp per curve writes the index of each of its
// tasks (fill tasks numbered first, contour tasks after them).
__global__ void k_task_map(int nc, const CurvePlan* __restrict__ plan, const DevState* __restrict__ st, int* tmap,
                           long long tcap, int ftile) {
  grid_dep_wait();
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= nc) return;
  const CurvePlan pl = plan[c];
  if (pl.kind == kNone) return;
  const int ntask = pl.kind == kFill ? fill_task_count(pl.nx, pl.ny, ftile) : (pl.count + kChunk - 1) / kChunk;
  const long long base = pl.kind == kFill ? pl.chunk_off : (long long)st->n_chunks + pl.chunk_off;
  for (int j = lane; j < ntask; j += 32) {
    const long long t = base + j;
    if (t < tcap) tmap[t] = c;
  }
}

template <int P>
__device__ void emit_contour(const ns_curves& cv, const CurveRef& cr, const float* U, const CurvePlan& pl, int l,
                             const ns_sample_params& sp, float o, float4& rec) {
  const float u = contour_u(pl, l, sp.kappa);
  const int i = find_span(U, P, cr.n, u);
  Eval<P> e;
  eval_curve<P>(reinterpret_cast<const float4*>(cv.key), cr, U, i, u, e);
  rec = make_float4(e.C[0], e.C[1], e.C[2] / sp.rho, o);
}

// Shape of a tangent-aligned contour Gaussian at sample l: {sigma_t, cos,
// sin, 0} with (cos, sin) = C'_xy/|C'_xy| (Eq. 2) and sigma_t = |C'_xy| du / rho,
// du = (b - a)/(M - 1) for open curves and (b - a)/M for closed ones (the
// parameter step between samples).  Where C'_xy vanishes the Gaussian stays
// isotropic: {sigma_n, 1, 0, 0}.  An isotropic contour set (contour_mode 0)
// gets {sigma_n, 1, 0, 0} everywhere.
template <int P>
__device__ float4 contour_shape(const ns_curves& cv, const CurveRef& cr, const float* U, const CurvePlan& pl, int l,
                                const ns_sample_params& sp) {
  const float u = contour_u(pl, l, sp.kappa);
  const int i = find_span(U, P, cr.n, u);
  Eval<P> e;
  eval_curve<P>(reinterpret_cast<const float4*>(cv.key), cr, U, i, u, e);
  const float sn = e.C[2] / sp.rho;
  if (sp.contour_mode != 1) return make_float4(sn, 1.f, 0.f, 0.f);
  float dN[P + 1];
  basis_deriv<P>(e.t, dN);
  float dS0 = 0.f, dS1 = 0.f, dW = 0.f;
#pragma unroll
  for (int k = 0; k <= P; ++k) {
    const float nw = dN[k] * e.cp[k].w;
    dS0 = fmaf(nw, e.cp[k].x, dS0);
    dS1 = fmaf(nw, e.cp[k].y, dS1);
    dW += nw;
  }
  const float iw = 1.f / e.W;
  const float vx = (dS0 - e.C[0] * dW) * iw, vy = (dS1 - e.C[1] * dW) * iw;
  const float n = sqrtf(vx * vx + vy * vy);
  if (!(n > 0.f)) return make_float4(sn, 1.f, 0.f, 0.f);
  const float step = (pl.b - pl.a) / float(pl.kind == kOpen ? pl.M - 1 : pl.M);
  return make_float4(n * step / sp.rho, vx / n, vy / n, 0.f);
}

__global__ void __launch_bounds__(256) k_emit_shape(ns_curves cv, ns_sample_params sp,
                                                    const CurvePlan* __restrict__ plan,
                                                    const float* __restrict__ knots,
                                                    const DevState* __restrict__ st,
                                                    const float4* __restrict__ rec, const int* __restrict__ gcurve,
                                                    float4* shape) {
  grid_dep_wait();
  const int G = st->g_count;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x) {
    const int c = gcurve[g];
    if (c < 0 || c >= cv.n_curves) continue;
    const CurvePlan pl = plan[c];
    if (pl.kind == kFill || pl.kind == kNone) {
      shape[g] = make_float4(rec[g].z, 1.f, 0.f, 0.f);
      continue;
    }
    const int l = g - pl.g_off;
    if (l < 0 || l >= pl.count) continue;
    const CurveRef cr = curve_ref(cv, c);
    const float* U = knots + cr.knot0;
    float4 sh = make_float4(rec[g].z, 1.f, 0.f, 0.f);
    NS_DISPATCH_P(cr.p, sh = contour_shape<P>(cv, cr, U, pl, l, sp));
    shape[g] = sh;
  }
}



// Distance from grid-local point q to the segment p0 -> p1 given as high and
// low parts {x_hi, y_hi, x_lo, y_lo} (Eq. S1): q - p0 and p1 - p0 are formed
// from the high parts first (exact for nearby points) and corrected by the
// low parts, so a point near the polyline gets its distance to about 1e-7 px.
// The projection parameter t takes the approximate quotient: at an interior
// optimum the distance is stationary in t, so its error enters only to second
// order; the distance takes the special-function unit's reciprocal square
// root (about 1e-7 relative).
__device__ __forceinline__ float seg_distance_hl(float qx, float qy, const float4& p0, const float4& p1) {
  const float rx = __fsub_rn(__fsub_rn(qx, p0.x), p0.z), ry = __fsub_rn(__fsub_rn(qy, p0.y), p0.w);
  const float ex = __fadd_rn(__fsub_rn(p1.x, p0.x), __fsub_rn(p1.z, p0.z));
  const float ey = __fadd_rn(__fsub_rn(p1.y, p0.y), __fsub_rn(p1.w, p0.w));
  const float ee = ex * ex + ey * ey;
  const float t = ee > 0.f ? fminf(fmaxf(__fdividef(rx * ex + ry * ey, ee), 0.f), 1.f) : 0.f;
  const float dx = rx - t * ex, dy = ry - t * ey;
  const float d2 = dx * dx + dy * dy;
  return d2 > 0.f ? d2 * rsqrtf(d2) : 0.f;
}

// Persistent over the contour tasks: each block iteration handles 256 samples
// of one open or closed stroke (Eq. 4-5).
__global__ void __launch_bounds__(256, 5) k_emit(ns_curves cv, ns_sample_params sp, const CurvePlan* __restrict__ plan,
                                              const int* __restrict__ order, const float* __restrict__ knots,
                                              const DevState* __restrict__ st, float4* rec, int* gcurve, int* gaux,
                                              long long gcap, const int* __restrict__ tmap, long long tcap) {
  grid_dep_wait();
  const int n_fill = st->n_chunks;
  const int n_tasks = st->n_ctasks;
  const int nc = cv.n_curves;
  for (int task = blockIdx.x; task < n_tasks; task += gridDim.x) {
    const int c = task_curve(tmap, tcap, n_fill, plan, order, nc, task, false);
    const CurvePlan pl = plan[c];
    if (pl.kind == kFill || pl.kind == kNone) continue;
    const CurveRef cr = curve_ref(cv, c);
    const float* U = knots + cr.knot0;
    const int l = (task - pl.chunk_off) * kChunk + threadIdx.x;
    const long long g = (long long)pl.g_off + l;
    if (l < pl.count && g < gcap) {
      float4 r;
      NS_DISPATCH_P(cr.p, emit_contour<P>(cv, cr, U, pl, l, sp, cv.color[4 * c + 3], r));
      rec[g] = r;
      gcurve[g] = c;
      gaux[g] = -1;
    }
  }
}

// ---------------------------------------------------------------------------
// Fill points (§3.3, Eq. 6-7 and S1-S3).  A fill point's opacity only needs
// the exact distance to the polyline inside a band around it: deeper inside,
// the sigmoid of Eq. 7 is exactly 1 in FP32 (R21), and farther outside the
// opacity stays below the cull threshold (R22).  So each task, a 16 x 16
// tile of one curve's grid, works from the segments instead of the points:
//   - the clusters of 8 segments whose boxes come within the band of the
//     tile list their segments, and every segment offers its distance to the
//     tile points within the band, kept per point as the smallest (squared
//     distance, segment index) by a 64-bit atomic minimum in shared memory --
//     the nearest segment of Eq. S1 with the lowest index among equal
//     distances, the same as a first-minimum loop over all segments;
//   - the segments that straddle a tile row are listed per row, and each point
//     counts their signed crossings of its ray to +x (Eq. S2, exact off the
//     polyline);
//   - a point in the band gets its distance recomputed from the high and low
//     parts of its nearest segment; a point outside it is deep (inside) or
//     culled (outside).  Where the band is not enough (no cull threshold, as at
//     the parity thresholds, or a cull distance beyond the band) an outside
//     point, and every point of a tile whose lists overflow, searches all
//     clusters with box lower bounds.
// All coordinates are grid-local (origin 0): the polyline's high parts.
constexpr int kRowX = 12;       // crossing segments listed per tile row

// Squared distance from q to segment {b0, e} (1/|e|^2 given), as in Eq. S1.
__device__ __forceinline__ float seg_d2(float qx, float qy, float4 sg, float inv_ee) {
  const float rx = qx - sg.x, ry = qy - sg.y;
  const float t = fminf(fmaxf((rx * sg.z + ry * sg.w) * inv_ee, 0.f), 1.f);
  const float dx = rx - t * sg.z, dy = ry - t * sg.w;
  return dx * dx + dy * dy;
}

// Segment k of a polyline of B points (high parts): {b0, b1 - b0}, b1.y, 1/|e|^2.
__device__ __forceinline__ float4 seg_at(const float4* __restrict__ bl, int B, int k, float& y1, float& inv_ee) {
  const float4 b0 = bl[k];
  const float4 b1 = bl[k + 1 == B ? 0 : k + 1];
  const float ex = b1.x - b0.x, ey = b1.y - b0.y;
  const float ee = ex * ex + ey * ey;
  inv_ee = ee > 0.f ? 1.f / ee : 0.f;
  y1 = b1.y;
  return make_float4(b0.x, b0.y, ex, ey);
}

// Signed crossing of segment {b0, e} (ending at height y1) by the ray from q to +x.
__device__ __forceinline__ int seg_crossing(float qx, float qy, float4 sg, float y1) {
  const float isleft = sg.z * (qy - sg.y) - (qx - sg.x) * sg.w;
  if (sg.y <= qy) return (y1 > qy && isleft > 0.f) ? 1 : 0;
  return (y1 <= qy && isleft < 0.f) ? -1 : 0;
}

// Nearest segment over the whole polyline (cluster boxes as lower bounds,
// lowest index among equal distances), and optionally the winding number.
__device__ void polyline_scan(const float4* __restrict__ bl, const float4* __restrict__ cb, int B, float qx, float qy,
                              bool want_d, float& best, int& arg, bool want_wn, int& wn) {
  const int ncl = (B + kCluster - 1) / kCluster;
  for (int cl = 0; cl < ncl; ++cl) {
    const float4 bb = cb[cl * kCluster];
    const int k1 = min(B, (cl + 1) * kCluster);
    const float bx = fmaxf(fmaxf(bb.x - qx, qx - bb.y), 0.f);
    const float by = fmaxf(fmaxf(bb.z - qy, qy - bb.w), 0.f);
    const float lb2 = bx * bx + by * by;
    const bool near = want_d && !(lb2 > best + 1e-3f * (lb2 + 1.f));
    const bool cross = want_wn && bb.z <= qy && bb.w > qy && bb.y >= qx - 0.01f;
    if (!near && !cross) continue;
    for (int k = cl * kCluster; k < k1; ++k) {
      float y1, inv_ee;
      const float4 sg = seg_at(bl, B, k, y1, inv_ee);
      if (near) {
        const float d2 = seg_d2(qx, qy, sg, inv_ee);
        if (d2 < best || (d2 == best && k < arg)) {
          best = d2;
          arg = k;
        }
      }
      if (cross) wn += seg_crossing(qx, qy, sg, y1);
    }
  }
}

constexpr int kSdfClaim = 2;   // fill tasks a block claims at a time

template <int TE>
__global__ void __launch_bounds__(TE * TE, 2048 / (TE * TE)) k_fill_sdf(ns_curves cv, ns_sample_params sp,
                                                     const CurvePlan* __restrict__ plan, const int* __restrict__ order,
                                                     const float4* __restrict__ bloc, const float2* __restrict__ glo,
                                                     const float4* __restrict__ cbox, DevState* st,
                                                     float4* rec, int* gcurve, int* gaux, long long gcap,
                                                     long long bcap, const int* __restrict__ tmap, long long tcap,
                                                     int4* lbox) {
  grid_dep_wait();
  // The lists and keys alternate between two buffers from task to task, so a
  // task takes two block barriers (after the lists, after the band): after
  // the first barrier of a task every thread is past the previous task's
  // points, and the previous task's buffer is cleared (its box added to its
  // curve's) for the task after this one, which writes it only after this
  // task's second barrier.
  // band segments listed per tile (a tile's band list beyond it falls back to
  // the search over the whole polyline): sized so that 2048 threads per SM fit
  constexpr int kNearCap = TE == 8 ? 64 : 256;
  __shared__ unsigned long long s_key[2][TE * TE];
  __shared__ float4 s_nseg[2][kNearCap];        // band segments {b0, e}
  __shared__ float2 s_ninfo[2][kNearCap];       // {index bits, 1/|e|^2}
  __shared__ float s_ny1[2][kNearCap];          // and their end heights
  __shared__ float4 s_xs[2][TE][kRowX];  // crossing segments per tile row {b0, e}
  __shared__ float s_xy1[2][TE][kRowX];  // and their end heights
  __shared__ int s_xcnt[2][TE];
  __shared__ int s_nnear[2];
  __shared__ int s_box[2][5];   // the tile's live box {min x, min y, max x, max y} and culled count
  const int n_fill = st->n_chunks;
  const int nc = cv.n_curves;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int b = 0; b < 2; ++b) {
    s_key[b][tid] = ~0ull;
    if (tid < TE) s_xcnt[b][tid] = 0;
    if (tid == 0) s_nnear[b] = 0;
    if (tid < 5) s_box[b][tid] = tid < 2 ? 0x7fffffff : (tid < 4 ? -1 : 0);
  }
  __syncthreads();
  int buf = 0;
  int prev_c = -1;   // the curve of the previous task, whose buffer (buf ^ 1) is not yet cleared
  // one thread adds a task's box of live grid points and culled count to its
  // curve's and resets the box
  auto flush_box = [&](int cc, int* box) {
    if (box[2] >= 0) {
      atomicMin(&lbox[cc].x, box[0]);
      atomicMin(&lbox[cc].y, box[1]);
      atomicMax(&lbox[cc].z, box[2]);
      atomicMax(&lbox[cc].w, box[3]);
    }
    if (box[4]) atomicAdd(&st->culled_s, (unsigned long long)box[4]);
    box[0] = box[1] = 0x7fffffff;
    box[2] = box[3] = -1;
    box[4] = 0;
  };
  // blocks claim runs of kSdfClaim consecutive tasks from a counter: the tiles
  // of a run mostly belong to one curve, whose polyline and cluster boxes then
  // stay in the SM's L1, and the claims balance the blocks' work
  __shared__ int s_claim;
  int task = 0, task_end = 0;
  for (;;) {
    if (task == task_end) {
      if (tid == 0) s_claim = atomicAdd(&st->sdf_next, kSdfClaim);
      __syncthreads();
      task = s_claim;
      task_end = min(n_fill, task + kSdfClaim);
      __syncthreads();   // s_claim is read by every thread before it is claimed again
      if (task >= n_fill) break;
    }
    const int c = task_curve(tmap, tcap, n_fill, plan, order, nc, task, true);
    const CurvePlan pl = plan[c];
    // a curve whose polyline did not fit the boundary capacity emits nothing
    // (block-uniform: the buffers stay as they are)
    if (pl.kind != kFill || (long long)pl.b_off + pl.M > bcap) {
      ++task;
      continue;
    }
    const int k = task - pl.chunk_off;
    int ix, iy;
    const bool in_grid = fill_task_point(k, pl.nx, pl.ny, tid, TE, ix, iy);
    const long long g = (long long)pl.g_off + (long long)iy * pl.nx + ix;
    const bool valid = in_grid && g < gcap;
    const int tix0 = ix - (tid % TE), tiy0 = iy - (tid / TE);   // the tile's first column and row
    const float h = sp.h, inv_h = 1.f / h;
    const float qx = (float(ix) + 0.5f) * h, qy = (float(iy) + 0.5f) * h;
    // the tile's point box
    const float tx0 = (float(tix0) + 0.5f) * h, tx1 = (float(min(pl.nx, tix0 + TE)) - 0.5f) * h;
    const float ty0 = (float(tiy0) + 0.5f) * h, ty1 = (float(min(pl.ny, tiy0 + TE)) - 0.5f) * h;
    const float o = cv.color[4 * c + 3];
    // sigmoid(z) rounds to exactly 1 in FP32 once exp(-z) <= 2^-24 (z >= 16.64);
    // deep2 is the squared distance beyond which z >= 17 with margin: the band
    const float dsat = 17.f * h / sp.gamma;
    const float deep2 = dsat * dsat * 1.001f + 1e-3f;
    const float band = sqrtf(deep2);
    const float near2 = deep2 * 1.001f + 1e-3f;   // box tests, with a margin for their rounding
    // outside, o sigmoid(-gamma d / h) < fill_cull once d > (h/gamma) ln(o/fill_cull - 1);
    // far2 adds a margin of 0.1 in z (FLT_MAX: no culling)
    float far2 = FLT_MAX;
    if (sp.fill_cull > 0.f && o > 1.01f * sp.fill_cull) {
      const float dcut = h / sp.gamma * (logf(o / sp.fill_cull - 1.f) + 0.1f);
      if (dcut > 0.f) far2 = dcut * dcut;
    }
    const float4* bl = bloc + pl.b_off;
    const float4* cb = cbox + pl.b_off;
    const int B = pl.M;
    // one thread per segment: segments of clusters whose boxes come within the
    // band of the tile join the band list, segments straddling a tile row to
    // the right of the tile's first column join that row's crossing list
    for (int kseg = tid; kseg < B; kseg += blockDim.x) {
      const float4 bb = cb[(kseg / kCluster) * kCluster];
      const float gx = fmaxf(fmaxf(bb.x - tx1, tx0 - bb.y), 0.f);
      const float gy = fmaxf(fmaxf(bb.z - ty1, ty0 - bb.w), 0.f);
      const bool ncl_near = gx * gx + gy * gy <= near2;
      const bool ncl_cross = bb.z <= ty1 && bb.w > ty0 && bb.y >= tx0 - 0.01f;
      if (!ncl_near && !ncl_cross) continue;
      float y1, inv_ee;
      const float4 sg = seg_at(bl, B, kseg, y1, inv_ee);
      const float xlo = fminf(sg.x, sg.x + sg.z), xhi = fmaxf(sg.x, sg.x + sg.z);
      const float ylo = fminf(sg.y, y1), yhi = fmaxf(sg.y, y1);
      if (ncl_near) {
        const float sx = fmaxf(fmaxf(xlo - tx1, tx0 - xhi), 0.f);
        const float sy = fmaxf(fmaxf(ylo - ty1, ty0 - yhi), 0.f);
        if (sx * sx + sy * sy <= near2) {
          const int slot = atomicAdd(&s_nnear[buf], 1);
          if (slot < kNearCap) {
            s_nseg[buf][slot] = sg;
            s_ninfo[buf][slot] = make_float2(__int_as_float(kseg), inv_ee);
            s_ny1[buf][slot] = y1;
          }
        }
      }
      if (ncl_cross && xhi >= tx0 - 0.01f) {
        // rows r of the tile with ylo <= qy_r < yhi (the straddle rule of the crossing test)
        // (row bounds from the reciprocal of h with a margin: each row is tested exactly)
        const int r0 = max(0, int(ceilf(ylo * inv_h - 0.5f - 1e-3f)) - tiy0 - 1);
        const int r1 = min(TE - 1, int(ceilf(yhi * inv_h - 0.5f + 1e-3f)) - tiy0);
        for (int r = r0; r <= r1; ++r) {
          const float qyr = (float(tiy0 + r) + 0.5f) * h;
          if (ylo <= qyr && qyr < yhi) {
            const int slot = atomicAdd(&s_xcnt[buf][r], 1);
            if (slot < kRowX) {
              s_xs[buf][r][slot] = sg;
              s_xy1[buf][r][slot] = y1;
            }
          }
        }
      }
    }
    __syncthreads();
    if (prev_c >= 0) {   // the previous task's buffer: flushed and cleared
      s_key[buf ^ 1][tid] = ~0ull;
      if (tid < TE) s_xcnt[buf ^ 1][tid] = 0;
      if (tid == 0) {
        s_nnear[buf ^ 1] = 0;
        flush_box(prev_c, s_box[buf ^ 1]);
      }
      prev_c = -1;
    }
    const int nnear = s_nnear[buf];
    const bool near_ovf = nnear > kNearCap;
    unsigned long long* key = s_key[buf];
    if (!near_ovf) {
      // band: one warp per listed segment, its lanes over the tile points
      // within the band of the segment's box
      for (int i = warp; i < nnear; i += blockDim.x >> 5) {
        const float4 sg = s_nseg[buf][i];
        const float2 info = s_ninfo[buf][i];
        const int kseg = __float_as_int(info.x);
        const float y1 = s_ny1[buf][i];
        const float xlo = fminf(sg.x, sg.x + sg.z) - band, xhi = fmaxf(sg.x, sg.x + sg.z) + band;
        const float ylo = fminf(sg.y, y1) - band, yhi = fmaxf(sg.y, y1) + band;
        // the band box in grid indices, from the reciprocal of h with a margin
        // of 1e-3 (points it adds are outside the band: the distance test
        // below rejects them)
        const int ia = max(tix0, int(ceilf(xlo * inv_h - 0.5f - 1e-3f)));
        const int ib = min(tix0 + TE - 1, int(floorf(xhi * inv_h - 0.5f + 1e-3f)));
        const int ja = max(tiy0, int(ceilf(ylo * inv_h - 0.5f - 1e-3f)));
        const int jb = min(tiy0 + TE - 1, int(floorf(yhi * inv_h - 0.5f + 1e-3f)));
        if (ia > ib || ja > jb) continue;
        const int w = ib - ia + 1, npts = w * (jb - ja + 1);
        const float inv_w = __fdividef(1.f, float(w));   // the quotients below stay 0.5/w off integers
        for (int p = lane; p < npts; p += 32) {
          const int py = int((float(p) + 0.5f) * inv_w);   // exact for the box sizes of a tile
          const int jx = ia + (p - py * w), jy = ja + py;
          const float d2 = seg_d2((float(jx) + 0.5f) * h, (float(jy) + 0.5f) * h, sg, info.y);
          if (d2 <= deep2)
            atomicMin(&key[(jy - tiy0) * TE + (jx - tix0)],
                      ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned int)kseg);
        }
      }
    }
    __syncthreads();
    bool live = false, culled = false;
    if (valid) {
      // winding number from the row's crossing list (or the whole polyline)
      int wn = 0;
      const int r = iy - tiy0;
      const int nx_r = s_xcnt[buf][r];
      if (nx_r <= kRowX) {
        for (int q = 0; q < nx_r; ++q) wn += seg_crossing(qx, qy, s_xs[buf][r][q], s_xy1[buf][r][q]);
      } else {
        float b_unused = FLT_MAX;
        int a_unused = 0;
        polyline_scan(bl, cb, B, qx, qy, false, b_unused, a_unused, true, wn);
      }
      const bool inside = sp.fill_rule == 0 ? wn > 0 : wn != 0;
      float best = FLT_MAX;
      int arg = 0;
      if (!near_ovf) {
        const unsigned long long kk = key[tid];
        if (kk != ~0ull) {
          best = __uint_as_float(unsigned(kk >> 32));
          arg = int(kk & 0xffffffffu);
        }
      }
      if (near_ovf || (!inside && best > deep2 && far2 > deep2)) {
        // an outside point beyond the band without a cull distance inside it,
        // or a tile whose band list overflowed: the exact nearest segment over
        // the whole polyline
        int w_unused = 0;
        best = FLT_MAX;
        arg = 0;
        polyline_scan(bl, cb, B, qx, qy, true, best, arg, false, w_unused);
      }
      const bool deep = inside && best > deep2;
      const bool far = !inside && best > far2;
      float sig = 1.f;
      if (far) {
        sig = 0.f;
      } else if (!deep) {
        const float d = seg_distance_hl(qx, qy, bl[arg], bl[arg + 1 == B ? 0 : arg + 1]);
        const float sdf = inside ? d : -d;
        const float z = sp.gamma * inv_h * sdf;
        sig = __fdividef(1.f, 1.f + __expf(-z));   // 0 once exp(-z) overflows
      }
      const float2 lo = glo[c];
      const float oj = o * sig;
      rec[g] = make_float4(__fadd_rn(pl.x0, __fadd_rn(qx, lo.x)), __fadd_rn(pl.y0, __fadd_rn(qy, lo.y)),
                           sp.eta * h / sp.rho, oj);
      gcurve[g] = c;
      gaux[g] = deep ? kAuxDeep : (far ? kAuxFar : (inside ? arg : ~arg));
      live = oj > 0.f && oj >= sp.fill_cull;   // sigma > 0 here
      culled = oj < sp.fill_cull;
    }
    {
      // the tile's box of live grid points and culled count (the rule the binning
      // applies for alpha_min = fill_cull): warps reduce, then shared atomics;
      // one thread adds the tile's to the curve's after the barrier
      const int bx0 = __reduce_min_sync(0xffffffffu, live ? ix : 0x7fffffff);
      const int by0 = __reduce_min_sync(0xffffffffu, live ? iy : 0x7fffffff);
      const int bx1 = __reduce_max_sync(0xffffffffu, live ? ix : -1);
      const int by1 = __reduce_max_sync(0xffffffffu, live ? iy : -1);
      const int nculled = __popc(__ballot_sync(0xffffffffu, culled));
      if (lane == 0) {
        if (bx1 >= 0) {
          atomicMin(&s_box[buf][0], bx0);
          atomicMin(&s_box[buf][1], by0);
          atomicMax(&s_box[buf][2], bx1);
          atomicMax(&s_box[buf][3], by1);
        }
        if (nculled) atomicAdd(&s_box[buf][4], nculled);
      }
    }
    prev_c = c;
    buf ^= 1;
    ++task;
  }
  // the last task's box (every thread is past its points: the claim that
  // ended the loop took two barriers)
  if (prev_c >= 0 && tid == 0) flush_box(prev_c, s_box[buf ^ 1]);
}

}  // namespace ns

using namespace ns;

extern "C" ns_status nurbs_sample(const ns_curves* curves, const ns_sample_params* sp, const ns_capacity* cap,
                                  const ns_gaussians* out, void* ws, size_t ws_bytes, void* stream) {
  Layout L;
  if (!curves || !sp || !cap || !out || !ws) {
    set_error("nurbs_sample: null argument");
    return NS_ERR_INVALID_ARG;
  }
  ns_raster_params rp = ns_default_raster_params();
  if (!make_layout(curves, cap, &rp, &L)) return NS_ERR_INVALID_ARG;
  if (ws_bytes < L.sample_total) {
    set_error("nurbs_sample: workspace too small");
    return NS_ERR_INVALID_ARG;
  }
  if (!(sp->h > 0.f) || !(sp->rho > 0.f) || !(sp->delta_c > 0.f) || !(sp->delta_b > 0.f) || sp->kappa < 0 ||
      sp->nl_mult < 1 || !(sp->eta > 0.f) || !(sp->pad_frac >= 0.f) || sp->fill_rule < 0 || sp->fill_rule > 1 ||
      (sp->fill_tile != 0 && sp->fill_tile != 8 && sp->fill_tile != 16)) {
    set_error("nurbs_sample: invalid sample parameters");
    return NS_ERR_INVALID_ARG;
  }
  if (out->capacity < cap->gaussians || !out->rec || !out->curve || !out->aux || !out->count) {
    set_error("nurbs_sample: output arrays missing or smaller than the Gaussian capacity");
    return NS_ERR_INVALID_ARG;
  }
  if (sp->contour_mode < 0 || sp->contour_mode > 1 || (sp->contour_mode == 1 && !out->shape)) {
    set_error("nurbs_sample: contour_mode must be 0 or 1, and 1 needs the Gaussian set's shape array");
    return NS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevState* st = at<DevState>(ws, L.o_state);
  CurvePlan* plan = at<CurvePlan>(ws, L.o_plan);
  float* knots = at<float>(ws, L.o_knots);
  int* order = at<int>(ws, L.o_order);
  float2* bpts = at<float2>(ws, L.o_bpts);
  const int nc = curves->n_curves;
  launch_reset_state(st, s, order, nc, out->count);   // also zeroes the order and the Gaussian count
  if (nc == 0) return cudaGetLastError() == cudaSuccess ? NS_OK : NS_ERR_CUDA;
  float2* krcp = at<float2>(ws, L.o_krcp);
  {
    // the plan: knot vectors and span forms, then arc lengths and counts
    // (one profiled range)
    float* forms = at<float>(ws, L.o_forms);
    ::ns::before_launch(NS_KERNEL_PLAN, s);
    launch_kernel(k_plan_forms, dim3(nc), dim3(kFormThreads), 0, s, *curves, plan, knots,
                  at<float>(ws, L.o_knots_lo), krcp, order, st, forms);
    ::ns::after_launch(-1, s);
    ::ns::before_launch(-1, s);
    launch_kernel(k_plan_length, dim3(nc), dim3(kPlanThreads), 0, s, *curves, *sp, plan,
                  static_cast<const float*>(knots), static_cast<const float*>(forms));
    ::ns::after_launch(NS_KERNEL_PLAN, s);
  }
  int* boffs = at<int>(ws, L.o_boffs);
  NS_LAUNCH(NS_KERNEL_SCAN, k_scan_boundary, 1, 1024, 0, s, nc, plan, st, cap->boundary, boffs);
  float4* bloc = at<float4>(ws, L.o_bloc);
  if (cap->boundary > 0)
    NS_LAUNCH(NS_KERNEL_BOUNDARY, k_boundary, int(std::min<long long>((cap->boundary + 255) / 256, num_sms() * 16LL)),
              256, 0, s, *curves, plan, knots, at<const float>(ws, L.o_knots_lo), krcp, st, bpts,
              at<int>(ws, L.o_bcurve),
              bloc, cap->boundary, static_cast<const int*>(boffs));
  int4* lbox = at<int4>(ws, L.o_lbox);
  float4* cbox = at<float4>(ws, L.o_cbox);
  NS_LAUNCH(NS_KERNEL_OTHER, k_boundary_box, (nc + 7) / 8, 256, 0, s, *curves, *sp, plan, knots, bloc,
            at<float2>(ws, L.o_glo), cap->boundary, lbox, st, cbox);
  const int ftile = fill_tile_of(sp->fill_tile);
  NS_LAUNCH(NS_KERNEL_SCAN, k_scan_gauss, 1, 1024, 0, s, nc, plan, order, st, cap->gaussians, out->count, ftile,
            at<int>(ws, L.o_bmix), (long long)L.bin_blocks);
  int* tmap = at<int>(ws, L.o_tasks);
  NS_LAUNCH(NS_KERNEL_SCAN, k_task_map, (nc + 7) / 8, 256, 0, s, nc, plan, st, tmap, (long long)L.tcap, ftile);
  const int grid = num_sms() * 8;
  // full occupancy (2048 threads per SM) needs most of the SM's shared memory
  static bool carveout = false;
  if (!carveout) {
    cudaFuncSetAttribute(k_fill_sdf<8>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         int(cudaSharedmemCarveoutMaxShared));
    cudaFuncSetAttribute(k_fill_sdf<16>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         int(cudaSharedmemCarveoutMaxShared));
    carveout = true;
  }
  if (ftile == 8)
    NS_LAUNCH(NS_KERNEL_FILL_SDF, k_fill_sdf<8>, num_sms() * 32, 64, 0, s, *curves, *sp, plan, order, bloc,
              at<const float2>(ws, L.o_glo), cbox, st, reinterpret_cast<float4*>(out->rec), out->curve, out->aux,
              cap->gaussians, cap->boundary, tmap, (long long)L.tcap, lbox);
  else
    NS_LAUNCH(NS_KERNEL_FILL_SDF, k_fill_sdf<16>, num_sms() * 8, 256, 0, s, *curves, *sp, plan, order, bloc,
              at<const float2>(ws, L.o_glo), cbox, st, reinterpret_cast<float4*>(out->rec), out->curve, out->aux,
              cap->gaussians, cap->boundary, tmap, (long long)L.tcap, lbox);
  // the strokes' samples (none when the caller's hint says the batch holds fills only)
  if (curves->stroke_degrees != 1)
    NS_LAUNCH(NS_KERNEL_EMIT, k_emit, grid, 256, 0, s, *curves, *sp, plan, order, knots, st,
              reinterpret_cast<float4*>(out->rec), out->curve, out->aux, cap->gaussians, tmap, (long long)L.tcap);
  else
    ::ns::empty_range(NS_KERNEL_EMIT, s);
  if (out->shape)
    NS_LAUNCH(NS_KERNEL_OTHER, k_emit_shape, grid, 256, 0, s, *curves, *sp, plan, knots, st,
              reinterpret_cast<const float4*>(out->rec), out->curve, reinterpret_cast<float4*>(out->shape));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("nurbs_sample: ") + cudaGetErrorString(e));
    return NS_ERR_CUDA;
  }
  return NS_OK;
}
