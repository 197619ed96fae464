// ns_geometry_loss: the geometric regularisers of the total loss (Eq. 10),
// with their gradients, on the plan and knots that nurbs_sample left in the
// workspace.
//
//   k_deriv_loss<P,R> Eq. 11: per curve the mean of |C^(r)_xy|^2 over N
//                    midpoint nodes u_j = a + (j + 1/2)(b - a)/N of the domain.
//                    C^(r) comes from the homogeneous curve S_h = sum N_i w_i
//                    (x_i, y_i, 1): its k-th derivative is a degree p-k
//                    B-spline, S_h^(k)(u) = sum_l N_{l,p-k}(u) Q^(k)_l with
//                    the derivative control points
//                      Q^(k)_l = (p-k+1)/(U_{l+p-k+1} - U_l) (Q^(k-1)_l - Q^(k-1)_{l-1}),
//                    and the lower-degree basis values are the levels of the
//                    span's Cox-de Boor triangle.  The quotient C = S/W is then
//                    differentiated by the Leibniz rule,
//                      C^(k) = (S^(k) - sum_{q=1..k} binom(k,q) W^(q) C^(k-q)) / W,
//                    which is Eq. 2 for k = 1.  The reverse sweep runs the same
//                    steps backwards into control points, weights and knots
//                    (the triangle's reverse sweep takes adjoints at every level).
//                    Each thread walks a run of consecutive nodes and keeps the
//                    span's gradients in registers until the span changes.
//   k_bbox_contour   Eq. 12 over the contour samples of strokes (the M sampled
//   k_bbox_boundary  centres, not the endpoint copies) and the boundary points
//                    of fills, both read from what nurbs_sample wrote: per axis
//                    phi(b_min - P) + phi(P - b_max), phi ReLU or softplus;
//                    where the slope is nonzero the gradient goes back through
//                    C(u).
//   k_knot_grads     (ns_backward.cu) turns the knot gradients into dtau.
#include <cuda_runtime.h>

#include "ns_internal.cuh"

namespace ns {

void launch_knot_grads(const ns_curves& cv, const CurvePlan* plan, const float* dknots, float* dtau,
                       cudaStream_t s);

constexpr int kMaxOrder = 4;       // highest derivative order of Eq. 11 supported
constexpr int kGeoCurveThreads = 128;
constexpr int kGeoMaxSpans = 256;  // curves with more spans take the per-node kernel
constexpr int kGeoStage = 256;     // knots and key points staged per curve

// Curves whose spans hold many nodes each (the Taylor forms' set-up is then
// shared by many nodes) and fit the per-curve shared memory take
// k_deriv_curve; the others the per-node kernel.
__device__ __forceinline__ bool taylor_path(const CurveRef& cr, int p, int nodes) {
  const int nspan = cr.n - p + 1;
  return nspan <= kGeoMaxSpans && cr.ntau + 2 * p + 1 <= kGeoStage && cr.nk <= kGeoStage && nodes >= 16 * nspan;
}
constexpr int kDerivRun = 8;       // quadrature nodes per thread
constexpr int kGeoThreads = 128;

struct GeoParams {
  float scale_d;      // lambda_deriv / (n_curves * nodes)
  int order, nodes;
  float lo[2], hi[2];
  float scale_b;      // lambda_bbox
  int penalty;        // NS_PENALTY_RELU / NS_PENALTY_SOFTPLUS
  int kappa;
  int freeze_w;       // rational weights frozen: no dL/dw is written
  int taylor;         // the per-curve Taylor kernels run (the batch's curves are short against the nodes)
};

// binomial coefficients up to k = kMaxP
__device__ __forceinline__ float binom_pascal(int k, int q) {
  const float row[kMaxP + 1][kMaxP + 1] = {{1, 0, 0, 0, 0, 0}, {1, 1, 0, 0, 0, 0}, {1, 2, 1, 0, 0, 0},
                                           {1, 3, 3, 1, 0, 0}, {1, 4, 6, 4, 1, 0}, {1, 5, 10, 10, 5, 1}};
  return row[k][q];
}

__device__ __forceinline__ float binom_small(int k, int q) {
  // binomial coefficients up to k = kMaxOrder
  const float row[kMaxOrder + 1][kMaxOrder + 1] = {
      {1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
  return row[k][q];
}

// N_{i-d+r, d}(u) from the span triangle (level P is the top row).
template <int P>
__device__ __forceinline__ float level_value(const Tri<P>& t, int d, int r) {
  return d == P ? t.N[r] : t.lev[d < P ? d : 0][r];
}

// Span-local accumulators of one thread's run of nodes.
template <int P>
struct SpanAcc {
  int span;
  float cp[P + 1][3];   // dL/d{x, y, w} of control points span-P .. span
  float kn[2 * P];      // dL/dU of knots span-P+1 .. span+P
};

template <int P>
__device__ __forceinline__ void acc_clear(SpanAcc<P>& a, int span) {
  a.span = span;
#pragma unroll
  for (int l = 0; l <= P; ++l) a.cp[l][0] = a.cp[l][1] = a.cp[l][2] = 0.f;
#pragma unroll
  for (int k = 0; k < 2 * P; ++k) a.kn[k] = 0.f;
}

// dknots NULL: knot intervals frozen, their gradients are dropped.
template <int P>
__device__ __forceinline__ void acc_flush(const CurveRef& cr, SpanAcc<P>& a, int freeze_w, float* dkey,
                                          float* dknots) {
  if (a.span < 0) return;
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    float* d = dkey + 4 * (long long)(cr.key0 + cp_to_key(a.span - P + l, P, cr.closed, cr.nk));
    if (a.cp[l][0] != 0.f) atomicAdd(d + 0, a.cp[l][0]);
    if (a.cp[l][1] != 0.f) atomicAdd(d + 1, a.cp[l][1]);
    if (!freeze_w && a.cp[l][2] != 0.f) atomicAdd(d + 3, a.cp[l][2]);
  }
  if (dknots) {
#pragma unroll
    for (int k = 0; k < 2 * P; ++k)
      if (a.kn[k] != 0.f) atomicAdd(dknots + cr.knot0 + a.span - P + 1 + k, a.kn[k]);
  }
}

// One quadrature node: returns |C^(R)_xy(u)|^2; with `acc` adds the gradient
// of scale * |C^(R)|^2 and returns dL/du in *du.
template <int P, int R>
__device__ float deriv_node(const float4* __restrict__ key, const CurveRef& cr, const float* __restrict__ U, int i,
                            float u, float scale, SpanAcc<P>* acc, float* du) {
  constexpr int r = R;
  constexpr int KM = P < kMaxOrder ? P : kMaxOrder;   // highest nonzero S_h derivative
  Tri<P> t;
  basis_fwd<P>(U, i, u, t);
  float4 q[P + 1];
  float Q[KM + 1][P + 1][3];
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    q[l] = key[cr.key0 + cp_to_key(i - P + l, P, cr.closed, cr.nk)];
    Q[0][l][0] = q[l].w * q[l].x;
    Q[0][l][1] = q[l].w * q[l].y;
    Q[0][l][2] = q[l].w;
  }
#pragma unroll
  for (int k = 1; k <= KM; ++k) {
    if (k > r) break;
#pragma unroll
    for (int l = k; l <= P; ++l) {
      // D >= U[i+1] - U[i] > 0: the interval [U_{i-P+l}, U_{i+l-k+1}] holds span i
      const float c = float(P - k + 1) / (U[i + l - k + 1] - U[i - P + l]);
#pragma unroll
      for (int e = 0; e < 3; ++e) Q[k][l][e] = c * (Q[k - 1][l][e] - Q[k - 1][l - 1][e]);
    }
  }
  // homogeneous derivatives H[k] = S_h^(k)(u), k = 0..r
  float H[kMaxOrder + 1][3];
#pragma unroll
  for (int k = 0; k <= kMaxOrder; ++k) {
    H[k][0] = H[k][1] = H[k][2] = 0.f;
    if (k <= r && k <= KM) {
#pragma unroll
      for (int l = k; l <= P; ++l) {
        const float n = level_value<P>(t, P - k, l - k);
#pragma unroll
        for (int e = 0; e < 3; ++e) H[k][e] = fmaf(n, Q[k][l][e], H[k][e]);
      }
    }
  }
  const float iw = 1.f / H[0][2];
  float Cd[kMaxOrder + 1][2];
#pragma unroll
  for (int k = 0; k <= kMaxOrder; ++k) {
    if (k > r) break;
    float ax = H[k][0], ay = H[k][1];
#pragma unroll
    for (int qq = 1; qq <= k; ++qq) {
      const float b = binom_small(k, qq) * H[qq][2];
      ax -= b * Cd[k - qq][0];
      ay -= b * Cd[k - qq][1];
    }
    Cd[k][0] = ax * iw;
    Cd[k][1] = ay * iw;
  }
  float cx = 0.f, cy = 0.f;
#pragma unroll
  for (int k = 0; k <= kMaxOrder; ++k)
    if (k == r) { cx = Cd[k][0]; cy = Cd[k][1]; }
  const float f = cx * cx + cy * cy;
  if (!acc) return f;

  // ---- reverse sweep
  float gC[kMaxOrder + 1][2];
  float gH[kMaxOrder + 1][3];
#pragma unroll
  for (int k = 0; k <= kMaxOrder; ++k) {
    gC[k][0] = gC[k][1] = 0.f;
    gH[k][0] = gH[k][1] = gH[k][2] = 0.f;
    if (k == r) {
      gC[k][0] = 2.f * scale * cx;
      gC[k][1] = 2.f * scale * cy;
    }
  }
#pragma unroll
  for (int k = kMaxOrder; k >= 0; --k) {
    if (k > r) continue;
    const float gx = gC[k][0] * iw, gy = gC[k][1] * iw;
    gH[k][0] += gx;
    gH[k][1] += gy;
    gH[0][2] -= gx * Cd[k][0] + gy * Cd[k][1];   // the division by W = H[0].w
#pragma unroll
    for (int qq = 1; qq <= k; ++qq) {
      const float b = binom_small(k, qq);
      gH[qq][2] -= b * (gx * Cd[k - qq][0] + gy * Cd[k - qq][1]);
      gC[k - qq][0] -= b * H[qq][2] * gx;
      gC[k - qq][1] -= b * H[qq][2] * gy;
    }
  }
  // H[k] = sum_l lev(P-k)[l-k] Q[k][l]: adjoints of the basis levels and of Q
  float gTop[P + 1];
  float gLow[P][P];
#pragma unroll
  for (int l = 0; l <= P; ++l) gTop[l] = 0.f;
#pragma unroll
  for (int d = 0; d < P; ++d)
#pragma unroll
    for (int l = 0; l < P; ++l) gLow[d][l] = 0.f;
  float gQ[P + 1][3];     // adjoint of Q[k] for the level being swept
#pragma unroll
  for (int l = 0; l <= P; ++l) gQ[l][0] = gQ[l][1] = gQ[l][2] = 0.f;
#pragma unroll
  for (int k = KM; k >= 0; --k) {
    if (k > r) continue;
    // contributions of H[k]
#pragma unroll
    for (int l = k; l <= P; ++l) {
      const float n = level_value<P>(t, P - k, l - k);
      const float gn = gH[k][0] * Q[k][l][0] + gH[k][1] * Q[k][l][1] + gH[k][2] * Q[k][l][2];
      if (k == 0) gTop[l] += gn; else gLow[P - k][l - k] += gn;
#pragma unroll
      for (int e = 0; e < 3; ++e) gQ[l][e] = fmaf(n, gH[k][e], gQ[l][e]);
    }
    if (k == 0) break;
    // Q[k][l] = c (Q[k-1][l] - Q[k-1][l-1]): hand the adjoint down one level
    float gPrev[P + 1][3];
#pragma unroll
    for (int l = 0; l <= P; ++l) gPrev[l][0] = gPrev[l][1] = gPrev[l][2] = 0.f;
#pragma unroll
    for (int l = k; l <= P; ++l) {
      const float D = U[i + l - k + 1] - U[i - P + l];
      const float c = float(P - k + 1) / D;
      float gc = 0.f;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        gPrev[l][e] += c * gQ[l][e];
        gPrev[l - 1][e] -= c * gQ[l][e];
        gc += gQ[l][e] * (Q[k - 1][l][e] - Q[k - 1][l - 1][e]);
      }
      const float gD = -gc * c / D;
      acc->kn[l - k + P] += gD;   // knot i+l-k+1
      acc->kn[l - 1] -= gD;       // knot i-P+l
    }
#pragma unroll
    for (int l = 0; l <= P; ++l) {
      gQ[l][0] = gPrev[l][0];
      gQ[l][1] = gPrev[l][1];
      gQ[l][2] = gPrev[l][2];
    }
  }
  // Q[0][l] = (w x, w y, w)
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    acc->cp[l][0] += q[l].w * gQ[l][0];
    acc->cp[l][1] += q[l].w * gQ[l][1];
    acc->cp[l][2] += q[l].x * gQ[l][0] + q[l].y * gQ[l][1] + gQ[l][2];
  }
  float d = 0.f;
  basis_bwd_levels<P>(t, gTop, gLow, &d, acc->kn);
  *du = d;
  return f;
}

template <int P, int R>
__device__ float deriv_run(const ns_curves& cv, const CurveRef& cr, const float* U, const CurvePlan& pl,
                           const GeoParams& gp, int j0, int j1, float* dkey, float* dknots) {
  SpanAcc<P> acc;
  const bool grads = dkey != nullptr;
  acc_clear<P>(acc, -1);
  float sum = 0.f, dA = 0.f, dB = 0.f;
  for (int j = j0; j < j1; ++j) {
    const float t = (float(j) + 0.5f) / float(gp.nodes);
    const float u = pl.a + t * (pl.b - pl.a);
    const int i = find_span(U, P, cr.n, u);
    if (grads && i != acc.span) {
      acc_flush<P>(cr, acc, gp.freeze_w, dkey, dknots);
      acc_clear<P>(acc, i);
    }
    float du = 0.f;
    sum += deriv_node<P, R>(reinterpret_cast<const float4*>(cv.key), cr, U, i, u, gp.scale_d,
                            grads ? &acc : nullptr, &du);
    dA += du * (1.f - t);   // u = a + t (b - a)
    dB += du * t;
  }
  if (grads) {
    acc_flush<P>(cr, acc, gp.freeze_w, dkey, dknots);
    if (dknots && dA != 0.f) atomicAdd(dknots + cr.knot0 + cr.p, dA);
    if (dknots && dB != 0.f) atomicAdd(dknots + cr.knot0 + cr.n + 1, dB);
  }
  return sum * gp.scale_d;
}

__device__ __forceinline__ void block_sum_add(float v, float* out) {
  __shared__ float s_part[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) s_part[w] = v;
  __syncthreads();
  if (w == 0) {
    float x = lane < int(blockDim.x >> 5) ? s_part[lane] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0 && x != 0.f) atomicAdd(out, x);
  }
}

// One kernel per (degree, order): each handles the curves of its degree (the
// degree-5 register count would otherwise set the occupancy of every curve).
template <int P, int R>
__global__ void __launch_bounds__(kGeoThreads) k_deriv_loss(ns_curves cv, const CurvePlan* __restrict__ plan,
                                                            const float* __restrict__ knots, GeoParams gp,
                                                            float* loss, float* dkey, float* dknots) {
  grid_dep_wait();
  const int runs = (gp.nodes + kDerivRun - 1) / kDerivRun;
  const long long total = (long long)cv.n_curves * runs;
  const long long stride = (long long)gridDim.x * blockDim.x;
  float sum = 0.f;
  // every thread runs the same number of iterations, so the block reduction
  // below is reached by all of them
  const long long iters = (total + stride - 1) / stride;
  for (long long it = 0; it < iters; ++it) {
    const long long idx = it * stride + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= total) continue;
    const int c = int(idx / runs);
    if (cv.degree[c] != P) continue;
    const int run = int(idx - (long long)c * runs);
    const CurvePlan pl = plan[c];
    if (pl.kind == kNone) continue;
    const CurveRef cr = curve_ref(cv, c);
    if (gp.taylor && taylor_path(cr, P, gp.nodes)) continue;   // done by k_deriv_curve
    const float* U = knots + cr.knot0;
    const int j0 = run * kDerivRun, j1 = min(j0 + kDerivRun, gp.nodes);
    sum += deriv_run<P, R>(cv, cr, U, pl, gp, j0, j1, dkey, dknots);
  }
  block_sum_add(sum, loss);
}

// ---------------------------------------------------------------------------
// Derivative loss per curve from the spans' Taylor forms.  One block per curve
// (with at most kGeoMaxSpans spans): the block builds every span's Taylor form
// S_h(u) = sum_k A[k] (u - m)^k once; each node then needs only the first r + 1
// derivatives of three polynomials (Horner with derivatives) and the Leibniz
// quotient.  The reverse sweep of a node stops at the span's coefficients A[k]
// and its centre m; the sums over the span's nodes then go once per span
// through the reverse of the Taylor form's construction (derivative control
// points and span triangle at m) into control points, weights and knots.
// Reverse of span_poly: gA[k][e] = dL/dA[k][e] and gm = dL/dm (from the nodes).
template <int P>
__device__ void span_poly_bwd(const float4* key, const CurveRef& cr, const float* U, int i, const float* gA,
                              float gm, float dcp[P + 1][3], float dkn[2 * P]) {
  const float m = 0.5f * (U[i] + U[i + 1]);
  Tri<P> t;
  basis_fwd<P>(U, i, m, t);
  float Q[P + 1][P + 1][3];
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    const float4 q = key[cr.key0 + cp_to_key(i - P + l, P, cr.closed, cr.nk)];
    Q[0][l][0] = q.w * q.x;
    Q[0][l][1] = q.w * q.y;
    Q[0][l][2] = q.w;
  }
#pragma unroll
  for (int k = 1; k <= P; ++k)
#pragma unroll
    for (int l = k; l <= P; ++l) {
      const float c = float(P - k + 1) / (U[i + l - k + 1] - U[i - P + l]);
#pragma unroll
      for (int e = 0; e < 3; ++e) Q[k][l][e] = c * (Q[k - 1][l][e] - Q[k - 1][l - 1][e]);
    }
  float gTop[P + 1];
  float gLow[P][P];
#pragma unroll
  for (int l = 0; l <= P; ++l) gTop[l] = 0.f;
#pragma unroll
  for (int d = 0; d < P; ++d)
#pragma unroll
    for (int l = 0; l < P; ++l) gLow[d][l] = 0.f;
  float gQ[P + 1][3];
#pragma unroll
  for (int l = 0; l <= P; ++l) gQ[l][0] = gQ[l][1] = gQ[l][2] = 0.f;
  float fact = 1.f;
#pragma unroll
  for (int k = 1; k <= P; ++k) fact *= float(k);   // P!
#pragma unroll
  for (int k = P; k >= 0; --k) {
    // A[k] = (1/k!) sum_l lev(P-k)[l-k] Q[k][l]
    const float inv = 1.f / fact;
    const float g0 = gA[3 * k] * inv, g1 = gA[3 * k + 1] * inv, g2 = gA[3 * k + 2] * inv;
#pragma unroll
    for (int l = k; l <= P; ++l) {
      const float n = (k == 0) ? t.N[l] : t.lev[P - k < P ? P - k : 0][l - k];
      const float gn = g0 * Q[k][l][0] + g1 * Q[k][l][1] + g2 * Q[k][l][2];
      if (k == 0) gTop[l] += gn; else gLow[P - k < P ? P - k : 0][l - k] += gn;
      gQ[l][0] = fmaf(n, g0, gQ[l][0]);
      gQ[l][1] = fmaf(n, g1, gQ[l][1]);
      gQ[l][2] = fmaf(n, g2, gQ[l][2]);
    }
    if (k > 0) fact /= float(k);
    if (k == 0) break;
    // Q[k][l] = c (Q[k-1][l] - Q[k-1][l-1])
    float gPrev[P + 1][3];
#pragma unroll
    for (int l = 0; l <= P; ++l) gPrev[l][0] = gPrev[l][1] = gPrev[l][2] = 0.f;
#pragma unroll
    for (int l = k; l <= P; ++l) {
      const float D = U[i + l - k + 1] - U[i - P + l];
      const float c = float(P - k + 1) / D;
      float gc = 0.f;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        gPrev[l][e] += c * gQ[l][e];
        gPrev[l - 1][e] -= c * gQ[l][e];
        gc += gQ[l][e] * (Q[k - 1][l][e] - Q[k - 1][l - 1][e]);
      }
      const float gD = -gc * c / D;
      dkn[l - k + P] += gD;   // knot i+l-k+1
      dkn[l - 1] -= gD;       // knot i-P+l
    }
#pragma unroll
    for (int l = 0; l <= P; ++l) {
      gQ[l][0] = gPrev[l][0];
      gQ[l][1] = gPrev[l][1];
      gQ[l][2] = gPrev[l][2];
    }
  }
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    const float4 q = key[cr.key0 + cp_to_key(i - P + l, P, cr.closed, cr.nk)];
    dcp[l][0] += q.w * gQ[l][0];
    dcp[l][1] += q.w * gQ[l][1];
    dcp[l][2] += q.x * gQ[l][0] + q.y * gQ[l][1] + gQ[l][2];
  }
  float dm = 0.f;
  basis_bwd_levels<P>(t, gTop, gLow, &dm, dkn);
  dm += gm;
  dkn[P - 1] += 0.5f * dm;   // m = (U_i + U_{i+1}) / 2
  dkn[P] += 0.5f * dm;
}

template <int P, int R>
__global__ void __launch_bounds__(kGeoCurveThreads) k_deriv_curve(ns_curves cv, const CurvePlan* __restrict__ plan,
                                                                  const float* __restrict__ knots, GeoParams gp,
                                                                  float* loss, float* dkey, float* dknots) {
  grid_dep_wait();
  constexpr int kPoly = 1 + 3 * (P + 1);   // {m, A[0..P][3]}
  constexpr int KD = R + 1;                // derivatives needed: up to R + 1 (the last for d/du)
  __shared__ float sU[kGeoStage];
  __shared__ float4 sK[kGeoStage];
  __shared__ float s_poly[kGeoMaxSpans * kPoly];
  __shared__ float s_grad[kGeoMaxSpans * kPoly];   // {dL/dm, dL/dA[0..P][3]} per span
  __shared__ float s_red[2];
  const int c = blockIdx.x;
  if (cv.degree[c] != P) return;
  const CurvePlan pl = plan[c];
  if (pl.kind == kNone) return;
  CurveRef cr = curve_ref(cv, c);
  const int nspan = cr.n - P + 1;
  const int nkn = cr.ntau + 2 * P + 1;
  if (!gp.taylor || !taylor_path(cr, P, gp.nodes)) return;   // left to k_deriv_loss
  const float* Ug = knots + cr.knot0;
  const float4* keyg = reinterpret_cast<const float4*>(cv.key) + cr.key0;
  for (int q = threadIdx.x; q < nkn; q += blockDim.x) sU[q] = Ug[q];
  for (int q = threadIdx.x; q < cr.nk; q += blockDim.x) sK[q] = keyg[q];
  for (int q = threadIdx.x; q < nspan * kPoly; q += blockDim.x) s_grad[q] = 0.f;
  if (threadIdx.x < 2) s_red[threadIdx.x] = 0.f;
  __syncthreads();
  const int key0 = cr.key0;
  cr.key0 = 0;   // key points now in sK
  for (int sidx = threadIdx.x; sidx < nspan; sidx += blockDim.x) {
    const int i = P + sidx;
    if (!(sU[i] < sU[i + 1])) continue;
    SpanPoly<P> sp;
    span_poly<P>(sK, cr, sU, i, sp);
    float* d = s_poly + sidx * kPoly;
    d[0] = sp.m;
#pragma unroll
    for (int k = 0; k <= P; ++k) {
      d[1 + 3 * k] = sp.A[k][0];
      d[2 + 3 * k] = sp.A[k][1];
      d[3 + 3 * k] = sp.A[k][2];
    }
  }
  __syncthreads();
  const bool grads = dkey != nullptr;
  const int N = gp.nodes;
  const int per = (N + blockDim.x - 1) / blockDim.x;
  const int j0 = threadIdx.x * per, j1 = min(N, j0 + per);
  float sum = 0.f, dA = 0.f, dB = 0.f;
  int span = -1;
  float hi = 0.f, m = 0.f;
  float A[P + 1][3], gAcc[P + 1][3], gmAcc = 0.f;
  auto flush = [&]() {
    if (!grads || span < 0) return;
    float* g = s_grad + (span - P) * kPoly;
    if (gmAcc != 0.f) atomicAdd(g, gmAcc);
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
      for (int e = 0; e < 3; ++e)
        if (gAcc[k][e] != 0.f) atomicAdd(g + 1 + 3 * k + e, gAcc[k][e]);
  };
  for (int j = j0; j < j1; ++j) {
    const float tn = (float(j) + 0.5f) / float(N);
    const float u = pl.a + tn * (pl.b - pl.a);
    if (span < 0 || !(u < hi)) {
      const int i = find_span(sU, P, cr.n, u);
      if (i != span) {
        flush();
        span = i;
        hi = i < cr.n ? sU[i + 1] : 3.0e38f;
        const float* d = s_poly + (i - P) * kPoly;
        m = d[0];
#pragma unroll
        for (int k = 0; k <= P; ++k) {
          A[k][0] = d[1 + 3 * k];
          A[k][1] = d[2 + 3 * k];
          A[k][2] = d[3 + 3 * k];
          gAcc[k][0] = gAcc[k][1] = gAcc[k][2] = 0.f;
        }
        gmAcc = 0.f;
      }
    }
    const float t = u - m;
    // Taylor coefficients at t: dd[e][q] = S_h^(q)(u) / q!, q = 0..KD
    float dd[3][KD + 1];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
#pragma unroll
      for (int q = 0; q <= KD; ++q) dd[e][q] = 0.f;
      dd[e][0] = A[P][e];
#pragma unroll
      for (int k = P - 1; k >= 0; --k) {
#pragma unroll
        for (int q = KD; q >= 1; --q)
          if (q <= P - k) dd[e][q] = fmaf(dd[e][q], t, dd[e][q - 1]);
        dd[e][0] = fmaf(dd[e][0], t, A[k][e]);
      }
    }
    // H[q] = S_h^(q), q = 0..R
    float H[R + 1][3];
    float qf = 1.f;
#pragma unroll
    for (int q = 0; q <= R; ++q) {
      if (q > 0) qf *= float(q);
#pragma unroll
      for (int e = 0; e < 3; ++e) H[q][e] = qf * dd[e][q];
    }
    const float iw = 1.f / H[0][2];
    float Cd[R + 1][2];
#pragma unroll
    for (int k = 0; k <= R; ++k) {
      float ax = H[k][0], ay = H[k][1];
#pragma unroll
      for (int q = 1; q <= k; ++q) {
        const float bq = binom_small(k, q) * H[q][2];
        ax -= bq * Cd[k - q][0];
        ay -= bq * Cd[k - q][1];
      }
      Cd[k][0] = ax * iw;
      Cd[k][1] = ay * iw;
    }
    const float cx = Cd[R][0], cy = Cd[R][1];
    sum += cx * cx + cy * cy;
    if (!grads) continue;
    // reverse of the Leibniz quotient -> gH[q][e]
    float gC[R + 1][2], gH[R + 1][3];
#pragma unroll
    for (int k = 0; k <= R; ++k) {
      gC[k][0] = gC[k][1] = 0.f;
      gH[k][0] = gH[k][1] = gH[k][2] = 0.f;
    }
    gC[R][0] = 2.f * gp.scale_d * cx;
    gC[R][1] = 2.f * gp.scale_d * cy;
#pragma unroll
    for (int k = R; k >= 0; --k) {
      const float gx = gC[k][0] * iw, gy = gC[k][1] * iw;
      gH[k][0] += gx;
      gH[k][1] += gy;
      gH[0][2] -= gx * Cd[k][0] + gy * Cd[k][1];
#pragma unroll
      for (int q = 1; q <= k; ++q) {
        const float bq = binom_small(k, q);
        gH[q][2] -= bq * (gx * Cd[k - q][0] + gy * Cd[k - q][1]);
        gC[k - q][0] -= bq * H[q][2] * gx;
        gC[k - q][1] -= bq * H[q][2] * gy;
      }
    }
    // H[q] = q! sum_k A[k] binom(k, q) t^(k-q): adjoints of A and of t (= of u)
    float gt = 0.f;
    qf = 1.f;
#pragma unroll
    for (int q = 0; q <= R; ++q) {
      if (q > 0) qf *= float(q);
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const float g = gH[q][e] * qf;   // dL/d dd[e][q]
        // dd[q] = sum_{k >= q} A[k] binom(k, q) t^(k-q); d dd[q]/dt = (q + 1) dd[q + 1]
        gt += g * float(q + 1) * dd[e][q + 1];
        float tp = 1.f;
#pragma unroll
        for (int k = q; k <= P; ++k) {
          gAcc[k][e] = fmaf(g * binom_pascal(k, q), tp, gAcc[k][e]);
          tp *= t;
        }
      }
    }
    gmAcc -= gt;                 // t = u - m
    dA += gt * (1.f - tn);       // u = a + tn (b - a)
    dB += gt * tn;
  }
  flush();
  // loss
  float v = sum * gp.scale_d;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0.f) atomicAdd(&s_red[0], v);
  __syncthreads();
  if (threadIdx.x == 0 && s_red[0] != 0.f) atomicAdd(loss, s_red[0]);
  if (!grads) return;
  // domain ends
  if (dknots) {
    float x = dA, y = dB;
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if ((threadIdx.x & 31) == 0) {
      if (x != 0.f) atomicAdd(dknots + cr.knot0 + P, x);
      if (y != 0.f) atomicAdd(dknots + cr.knot0 + cr.n + 1, y);
    }
  }
  // each span: the reverse of its Taylor form's construction
  for (int sidx = threadIdx.x; sidx < nspan; sidx += blockDim.x) {
    const int i = P + sidx;
    if (!(sU[i] < sU[i + 1])) continue;
    const float* g = s_grad + sidx * kPoly;
    float dcp[P + 1][3], dkn[2 * P];
#pragma unroll
    for (int l = 0; l <= P; ++l) dcp[l][0] = dcp[l][1] = dcp[l][2] = 0.f;
#pragma unroll
    for (int q = 0; q < 2 * P; ++q) dkn[q] = 0.f;
    span_poly_bwd<P>(sK, cr, sU, i, g + 1, g[0], dcp, dkn);
#pragma unroll
    for (int l = 0; l <= P; ++l) {
      float* dk = dkey + 4 * (long long)(key0 + cp_to_key(i - P + l, P, cr.closed, cr.nk));
      if (dcp[l][0] != 0.f) atomicAdd(dk + 0, dcp[l][0]);
      if (dcp[l][1] != 0.f) atomicAdd(dk + 1, dcp[l][1]);
      if (!gp.freeze_w && dcp[l][2] != 0.f) atomicAdd(dk + 3, dcp[l][2]);
    }
    if (dknots)
#pragma unroll
      for (int q = 0; q < 2 * P; ++q)
        if (dkn[q] != 0.f) atomicAdd(dknots + cr.knot0 + i - P + 1 + q, dkn[q]);
  }
}

template <int R>
void launch_deriv_loss(const ns_curves& cv, const CurvePlan* plan, const float* knots, const GeoParams& gp,
                       float* loss, float* dkey, float* dknots, cudaStream_t s) {
  const int grid = num_sms() * 8;
  // the five launches form one profiled range (armed events bracket the first
  // and the last)
  auto run = [&](void (*k)(ns_curves, const CurvePlan*, const float*, GeoParams, float*, float*, float*),
                 int first_id, int last_id) {
    before_launch(first_id, s);
    k<<<grid, kGeoThreads, 0, s>>>(cv, plan, knots, gp, loss, dkey, dknots);
    after_launch(last_id, s);
  };
  auto run_curve = [&](void (*k)(ns_curves, const CurvePlan*, const float*, GeoParams, float*, float*, float*),
                       int first_id, int last_id) {
    before_launch(first_id, s);
    k<<<cv.n_curves, kGeoCurveThreads, 0, s>>>(cv, plan, knots, gp, loss, dkey, dknots);
    after_launch(last_id, s);
  };
  // curves within the shared-memory limits with many nodes per span: one block
  // each, per degree (launched only when the batch's mean key count makes that
  // the common case); the others: per-node kernels
  if (gp.taylor) {
    run_curve(k_deriv_curve<1, R>, NS_KERNEL_DERIV_LOSS, -1);
    run_curve(k_deriv_curve<2, R>, -1, -1);
    run_curve(k_deriv_curve<3, R>, -1, -1);
    run_curve(k_deriv_curve<4, R>, -1, -1);
    run_curve(k_deriv_curve<5, R>, -1, -1);
  }
  run(k_deriv_loss<1, R>, gp.taylor ? -1 : NS_KERNEL_DERIV_LOSS, -1);
  run(k_deriv_loss<2, R>, -1, -1);
  run(k_deriv_loss<3, R>, -1, -1);
  run(k_deriv_loss<4, R>, -1, -1);
  run(k_deriv_loss<5, R>, -1, NS_KERNEL_DERIV_LOSS);
}

// Penalty of one point and its gradient dL/dP (before the lambda scale).
__device__ __forceinline__ float box_penalty(const GeoParams& gp, float x, float y, float* gx, float* gy) {
  const float v[4] = {gp.lo[0] - x, gp.lo[1] - y, x - gp.hi[0], y - gp.hi[1]};
  float f = 0.f, d[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (gp.penalty == NS_PENALTY_SOFTPLUS) {
      // log(1 + e^v) = max(v, 0) + log(1 + e^-|v|), derivative the logistic function
      f += fmaxf(v[k], 0.f) + log1pf(expf(-fabsf(v[k])));
      d[k] = 1.f / (1.f + expf(-v[k]));
    } else {
      f += fmaxf(v[k], 0.f);
      d[k] = v[k] > 0.f ? 1.f : 0.f;
    }
  }
  *gx = d[2] - d[0];
  *gy = d[3] - d[1];
  return f;
}

// Gradient of the penalty at one curve point C(u), u = a + t (b - a): back
// through C(u) (Eq. 1) into control points, weights and knots.
template <int P>
__device__ void bbox_grad(const ns_curves& cv, const CurveRef& cr, const float* U, float u, float t, float gx,
                          float gy, int freeze_w, float* dkey, float* dknots) {
  const int i = find_span(U, P, cr.n, u);
  Eval<P> e;
  eval_curve<P>(reinterpret_cast<const float4*>(cv.key), cr, U, i, u, e);
  const float gC[3] = {gx, gy, 0.f};
  float dcp[P + 1][4], dkn[2 * P], du = 0.f;
#pragma unroll
  for (int l = 0; l <= P; ++l) dcp[l][0] = dcp[l][1] = dcp[l][2] = dcp[l][3] = 0.f;
#pragma unroll
  for (int k = 0; k < 2 * P; ++k) dkn[k] = 0.f;
  curve_point_adjoint<P>(e, gC, dcp, dkn, &du);
#pragma unroll
  for (int l = 0; l <= P; ++l) {
    float* d = dkey + 4 * (long long)(cr.key0 + cp_to_key(i - P + l, P, cr.closed, cr.nk));
    if (dcp[l][0] != 0.f) atomicAdd(d + 0, dcp[l][0]);
    if (dcp[l][1] != 0.f) atomicAdd(d + 1, dcp[l][1]);
    if (!freeze_w && dcp[l][3] != 0.f) atomicAdd(d + 3, dcp[l][3]);
  }
  if (!dknots) return;
#pragma unroll
  for (int k = 0; k < 2 * P; ++k)
    if (dkn[k] != 0.f) atomicAdd(dknots + cr.knot0 + i - P + 1 + k, dkn[k]);
  const float dA = du * (1.f - t), dB = du * t;
  if (dA != 0.f) atomicAdd(dknots + cr.knot0 + cr.p, dA);
  if (dB != 0.f) atomicAdd(dknots + cr.knot0 + cr.n + 1, dB);
}

// Contour samples of strokes, read from the sampled records: a contour
// Gaussian's centre is C(u_j) (Eq. 4).  Fill Gaussians and the endpoint
// copies of open curves are skipped.
__global__ void __launch_bounds__(kGeoThreads) k_bbox_contour(ns_curves cv, const CurvePlan* __restrict__ plan,
                                                              const float* __restrict__ knots,
                                                              const float4* __restrict__ rec,
                                                              const int* __restrict__ gcurve,
                                                              const int* __restrict__ gcount, GeoParams gp,
                                                              float* loss, float* dkey, float* dknots) {
  grid_dep_wait();
  const int n = *gcount;
  const int nc = cv.n_curves;
  const int stride = gridDim.x * blockDim.x;
  const int iters = (n + stride - 1) / stride;
  float sum = 0.f;
  for (int it = 0; it < iters; ++it) {
    const int gi = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= n) continue;
    const int c = gcurve[gi];
    if (c < 0 || c >= nc) continue;
    const CurvePlan& pl = plan[c];
    const int kind = pl.kind;
    if (kind != kOpen && kind != kClosedStroke) continue;
    const int l = gi - pl.g_off;
    if (l < 0 || l >= pl.count) continue;
    if (kind == kOpen && (l < gp.kappa || l >= gp.kappa + pl.M)) continue;   // endpoint copies
    const float4 r = rec[gi];
    float gx, gy;
    sum += box_penalty(gp, r.x, r.y, &gx, &gy);
    if (dkey && (gx != 0.f || gy != 0.f)) {
      const CurvePlan q = pl;
      const CurveRef cr = curve_ref(cv, c);
      const float* U = knots + cr.knot0;
      const float t = contour_t(q, l, gp.kappa);
      const float u = contour_u(q, l, gp.kappa);
      NS_DISPATCH_P(cr.p, bbox_grad<P>(cv, cr, U, u, t, gp.scale_b * gx, gp.scale_b * gy, gp.freeze_w, dkey, dknots));
    }
  }
  block_sum_add(sum * gp.scale_b, loss);
}

// Boundary points of filled curves, read from the polyline nurbs_sample built.
__global__ void __launch_bounds__(kGeoThreads) k_bbox_boundary(ns_curves cv, const CurvePlan* __restrict__ plan,
                                                               const float* __restrict__ knots,
                                                               const float2* __restrict__ bpts,
                                                               const int* __restrict__ bcurve,
                                                               const DevState* __restrict__ st, GeoParams gp,
                                                               float* loss, float* dkey, float* dknots) {
  grid_dep_wait();
  const int nb = st->b_count;
  const int nc = cv.n_curves;
  const int stride = gridDim.x * blockDim.x;
  const int iters = (nb + stride - 1) / stride;
  float sum = 0.f;
  for (int it = 0; it < iters; ++it) {
    const int j = it * stride + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nb) continue;
    const float2 b = bpts[j];
    float gx, gy;
    sum += box_penalty(gp, b.x, b.y, &gx, &gy);
    if (!dkey || (gx == 0.f && gy == 0.f)) continue;
    const int lo = bcurve[j];   // the curve that owns boundary point j
    if (lo < 0 || lo >= nc) continue;
    const CurvePlan pl = plan[lo];
    const int jj = j - pl.b_off;
    if (pl.kind != kFill || jj >= pl.M) continue;
    const CurveRef cr = curve_ref(cv, lo);
    const float* U = knots + cr.knot0;
    const float t = float(jj) / float(pl.M);
    const float u = pl.a + t * (pl.b - pl.a);
    NS_DISPATCH_P(cr.p, bbox_grad<P>(cv, cr, U, u, t, gp.scale_b * gx, gp.scale_b * gy, gp.freeze_w, dkey, dknots));
  }
  block_sum_add(sum * gp.scale_b, loss);
}

}  // namespace ns

using namespace ns;

extern "C" ns_geometry_params ns_default_geometry_params(void) {
  ns_geometry_params g;
  g.lambda_deriv = 1.f;
  g.order = 3;
  g.nodes = 0;
  g.lambda_bbox = 5.f;
  g.penalty = NS_PENALTY_RELU;
  g.box[0] = g.box[1] = g.box[2] = g.box[3] = 0.f;
  return g;
}

extern "C" ns_status ns_geometry_loss(const ns_curves* curves, const ns_gaussians* g, const ns_sample_params* sp,
                                      const ns_raster_params* rp, const ns_geometry_params* gpar,
                                      const ns_capacity* cap, float* loss, const ns_curve_grads* out,
                                      void* ws, size_t ws_bytes, void* stream) {
  if (!curves || !g || !sp || !rp || !gpar || !cap || !loss || !ws) {
    set_error("ns_geometry_loss: null argument");
    return NS_ERR_INVALID_ARG;
  }
  const bool knots_on = out && !(out->frozen & NS_FROZEN_KNOTS);
  if (out && (!out->dkey || (knots_on && !out->dtau))) {
    set_error("ns_geometry_loss: gradients need dkey and (unless the knots are frozen) dtau");
    return NS_ERR_INVALID_ARG;
  }
  if (gpar->order < 1 || gpar->order > kMaxOrder) {
    set_error("ns_geometry_loss: order must be 1..4");
    return NS_ERR_INVALID_ARG;
  }
  if (gpar->penalty != NS_PENALTY_RELU && gpar->penalty != NS_PENALTY_SOFTPLUS) {
    set_error("ns_geometry_loss: penalty must be NS_PENALTY_RELU or NS_PENALTY_SOFTPLUS");
    return NS_ERR_INVALID_ARG;
  }
  if (gpar->nodes < 0 || sp->nl_mult < 1 || sp->kappa < 0) {
    set_error("ns_geometry_loss: nodes must be >= 0 (0: N_L), nl_mult >= 1, kappa >= 0");
    return NS_ERR_INVALID_ARG;
  }
  Layout L;
  if (!make_layout(curves, cap, rp, &L)) return NS_ERR_INVALID_ARG;
  if (ws_bytes < L.total) {
    set_error("ns_geometry_loss: workspace smaller than ns_workspace_size");
    return NS_ERR_INVALID_ARG;
  }
  if (gpar->lambda_bbox != 0.f && (!g->rec || !g->curve || !g->count)) {
    set_error("ns_geometry_loss: the box loss reads the Gaussian records, curves and count");
    return NS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaMemsetAsync(loss, 0, 2 * sizeof(float), s);
  if (L.nc > 0) {
    GeoParams gp;
    gp.order = gpar->order;
    gp.nodes = gpar->nodes > 0 ? gpar->nodes : sp->nl_mult * (L.W > L.H ? L.W : L.H);
    gp.scale_d = gpar->lambda_deriv / (float(L.nc) * float(gp.nodes));
    const bool canvas = !(gpar->box[2] > gpar->box[0] && gpar->box[3] > gpar->box[1]);
    gp.lo[0] = canvas ? 0.f : gpar->box[0];
    gp.lo[1] = canvas ? 0.f : gpar->box[1];
    gp.hi[0] = canvas ? float(L.W) : gpar->box[2];
    gp.hi[1] = canvas ? float(L.H) : gpar->box[3];
    gp.scale_b = gpar->lambda_bbox;
    gp.penalty = gpar->penalty;
    gp.kappa = sp->kappa;
    gp.freeze_w = out && (out->frozen & NS_FROZEN_WEIGHTS) != 0;
    // the per-curve Taylor kernels pay off when spans hold many nodes: decided
    // from the batch's mean key count
    gp.taylor = (long long)gp.nodes >= 16LL * ((long long)L.nk / L.nc + 6);
    const CurvePlan* plan = at<const CurvePlan>(ws, L.o_plan);
    const float* knots = at<const float>(ws, L.o_knots);
    const DevState* st = at<const DevState>(ws, L.o_state);
    float* dknots = knots_on ? at<float>(ws, L.o_dknots) : nullptr;
    float* dkey = out ? out->dkey : nullptr;
    if (knots_on) cudaMemsetAsync(dknots, 0, sizeof(float) * ((size_t)L.nt + (size_t)kKnotPad * L.nc), s);
    if (gpar->lambda_deriv != 0.f) {
      switch (gp.order) {
        case 1: launch_deriv_loss<1>(*curves, plan, knots, gp, loss, dkey, dknots, s); break;
        case 2: launch_deriv_loss<2>(*curves, plan, knots, gp, loss, dkey, dknots, s); break;
        case 3: launch_deriv_loss<3>(*curves, plan, knots, gp, loss, dkey, dknots, s); break;
        default: launch_deriv_loss<4>(*curves, plan, knots, gp, loss, dkey, dknots, s); break;
      }
    }
    if (gpar->lambda_bbox != 0.f) {
      // the two launches form one profiled range
      const int grid = num_sms() * 8;
      before_launch(NS_KERNEL_BBOX_LOSS, s);
      k_bbox_contour<<<grid, kGeoThreads, 0, s>>>(*curves, plan, knots, reinterpret_cast<const float4*>(g->rec),
                                                  g->curve, g->count, gp, loss + 1, dkey, dknots);
      after_launch(-1, s);
      before_launch(-1, s);
      k_bbox_boundary<<<grid, kGeoThreads, 0, s>>>(*curves, plan, knots, at<const float2>(ws, L.o_bpts),
                                                   at<const int>(ws, L.o_bcurve), st, gp, loss + 1, dkey, dknots);
      after_launch(NS_KERNEL_BBOX_LOSS, s);
    }
    if (knots_on) launch_knot_grads(*curves, plan, dknots, out->dtau, s);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("ns_geometry_loss: ") + cudaGetErrorString(e));
    return NS_ERR_CUDA;
  }
  return NS_OK;
}
