// splat_forward and the blend adjoint: Gaussians -> image (paper §3.4, Eq. 8-9).
//
// Kernels, in launch order:
//   k_curve_scene   scene of every curve (binary search of the scene offsets)
//   k_bin_count     per 2048 Gaussians: tiles overlapped by mu +- k sigma (exact
//                   float32 rule), block sums; with fill layers, the live box
//                   of every filled curve's grid
//   k_layer_count   fill layers: each layer's tile count joins its block's sum
//   k_scan_small    one block: block sums -> block offsets, pair total; zeroes
//                   the radix sort's digit totals
//   k_layer_emit    fill layers whose first Gaussian lies in a block of fill
//                   Gaussians only: their pairs, one block per curve
//   k_bin_emit      recount, block-local scan, write (tile, Gaussian) pairs in
//                   Gaussian order, which is front to back inside each scene
//                   (a fill layer: one pair per tile of its live grid box)
//   k_layer_runs    fill layers: per curve and tile column (row), the grid
//                   columns (rows) the bin rule puts on it, and the layer's
//                   constants
//   k_radix_hist / k_radix_scan / k_radix_scatter
//                   stable LSD radix sort of the pairs on the tile id bits
//                   (per pass: digit counts per block of 4096 pairs and the
//                   digit totals, their scan, the stable scatter)
//                   only: pairs enter in (layer, sample) order, so a stable sort
//                   by tile yields the full (tile, layer, sample) order
//   k_ranges        [start, end) of every tile's run
//   k_blend_fwd     one tile per block, one 8 x 4 PPT sub-block per warp: each
//                   warp streams its tile's list 32 entries at a time, culls by
//                   ballot the entries that cannot reach its sub-block, and each
//                   thread composites its pixels front to back; a warp stops
//                   once all its pixels are done
//   k_blend_bwd     the adjoint, back to front from each pixel's last
//                   composited entry, transmittance recovered by division,
//                   warp-reduced per-Gaussian gradients
//   k_blend_fwd_groups / k_blend_bwd_groups
//                   the same with each warp split into four 8-lane groups of
//                   two pixel columns, each group walking its own hits
//   k_blend_fwd_layers / k_blend_bwd_layers
//                   the same lists where a fill layer's entry is walked as its
//                   grid: each warp stages the grid points its pixels can see
#include <cuda_runtime.h>

#include <algorithm>
#include <float.h>

#include "ns_internal.cuh"

namespace ns {


// The scene of every curve, and what the forward clears before it
// accumulates (in this launch instead of a memset each): the forward's
// counters, the tile ranges, and with fill layers (lmin != NULL) the live
// extremes of every curve's layer (lmin above every index, lmax -1).
__global__ void k_curve_scene(ns_curves cv, int* curve_scene, DevState* st, int2* ranges, int n_tiles, int2* lmin,
                              int2* lmax) {
  grid_dep_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    st->culled = 0;
    st->blend_evals = 0;
    st->blend_contribs = 0;
    st->blend_visits = 0;
  }
  for (int i = t; i < n_tiles; i += gridDim.x * blockDim.x) ranges[i] = make_int2(0, 0);
  const int c = t;
  if (c >= cv.n_curves) return;
  if (lmin) {
    lmin[c] = make_int2(0x7f7f7f7f, 0x7f7f7f7f);
    lmax[c] = make_int2(-1, -1);
  }
  int s = 0;
  if (cv.scene_curve_offset) {
    int lo = 0, hi = cv.n_scenes - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (cv.scene_curve_offset[mid] <= c) lo = mid; else hi = mid - 1;
    }
    s = lo;
  }
  curve_scene[c] = s;
}

struct BinParams {
  float k_sigma, inv_tile, alpha_min, log_amin;   // log_amin = ln(alpha_min), or -inf
  int tiles_x, tiles_y, tiles_per_scene;
  int n_curves, gcap;   // Gaussians naming a curve outside [0, n_curves) cover no tile
  int fill_layers;      // one pair per (tile, filled curve) instead of per (tile, Gaussian)
  int2* lmin;           // fill layers: per curve the smallest / largest grid column and row of a
  int2* lmax;           // live Gaussian (one the per-Gaussian rule would bin); empty: lmax < lmin
  // fill layers with nurbs_sample's live boxes (when its threshold is alpha_min): the boxes,
  // per binning block whether it holds a Gaussian outside the fill layers, per curve its
  // layer's pair count
  const int4* lbox;
  const int* bmix;   // per binning block: 1 if a stroke's Gaussian lies in it (nurbs_sample)
  int* bflag;
  int* lcount;
};

// Whether the binning may take nurbs_sample's live boxes and culled count:
// fill layers, and the sampling counted for this alpha_min.
__device__ __forceinline__ bool sampled_boxes(const BinParams& bp, const DevState* st) {
  return bp.fill_layers && st->cull_thr == bp.alpha_min;
}

// Pair values of fill layers carry this bit on the index of the layer's first Gaussian.
constexpr uint32_t kLayerBit = 0x80000000u;

// Tile rectangle of one Gaussian; every step one float32 operation rounded to
// nearest so that the result is reproducible bit for bit.
__device__ __forceinline__ int tile_rect(const float4 r, const BinParams& bp, int& x0, int& y0, int& nx) {
  const float ks = __fmul_rn(bp.k_sigma, r.z);
  const float xlo = floorf(__fmul_rn(__fsub_rn(r.x, ks), bp.inv_tile));
  const float xhi = floorf(__fmul_rn(__fadd_rn(r.x, ks), bp.inv_tile));
  const float ylo = floorf(__fmul_rn(__fsub_rn(r.y, ks), bp.inv_tile));
  const float yhi = floorf(__fmul_rn(__fadd_rn(r.y, ks), bp.inv_tile));
  const bool ok = r.z > 0.f && r.w > 0.f && r.w >= bp.alpha_min && xhi >= 0.f && yhi >= 0.f &&
                  xlo <= float(bp.tiles_x - 1) && ylo <= float(bp.tiles_y - 1);
  if (!ok) return 0;
  x0 = int(fmaxf(xlo, 0.f));
  const int x1 = int(fminf(xhi, float(bp.tiles_x - 1)));
  y0 = int(fmaxf(ylo, 0.f));
  const int y1 = int(fminf(yhi, float(bp.tiles_y - 1)));
  nx = x1 - x0 + 1;
  return nx * (y1 - y0 + 1);
}

// The same for a tangent-aligned Gaussian, sh = {sigma_t, cos, sin, 0} and
// r.z = sigma_n: the half widths of the k_sigma ellipse's bounding box,
// k sqrt(sigma_t^2 c^2 + sigma_n^2 s^2) in x and k sqrt(sigma_t^2 s^2 + sigma_n^2 c^2)
// in y, each operation rounded to nearest in this order.
__device__ __forceinline__ int tile_rect_aniso(const float4 r, const float4 sh, const BinParams& bp, int& x0,
                                               int& y0, int& nx) {
  const float st2 = __fmul_rn(sh.x, sh.x), cs2 = __fmul_rn(sh.y, sh.y), sn2 = __fmul_rn(sh.z, sh.z);
  const float sg2 = __fmul_rn(r.z, r.z);
  const float kx = __fmul_rn(bp.k_sigma, __fsqrt_rn(__fadd_rn(__fmul_rn(st2, cs2), __fmul_rn(sg2, sn2))));
  const float ky = __fmul_rn(bp.k_sigma, __fsqrt_rn(__fadd_rn(__fmul_rn(st2, sn2), __fmul_rn(sg2, cs2))));
  const float xlo = floorf(__fmul_rn(__fsub_rn(r.x, kx), bp.inv_tile));
  const float xhi = floorf(__fmul_rn(__fadd_rn(r.x, kx), bp.inv_tile));
  const float ylo = floorf(__fmul_rn(__fsub_rn(r.y, ky), bp.inv_tile));
  const float yhi = floorf(__fmul_rn(__fadd_rn(r.y, ky), bp.inv_tile));
  const bool ok = r.z > 0.f && sh.x > 0.f && r.w > 0.f && r.w >= bp.alpha_min && xhi >= 0.f && yhi >= 0.f &&
                  xlo <= float(bp.tiles_x - 1) && ylo <= float(bp.tiles_y - 1);
  if (!ok) return 0;
  x0 = int(fmaxf(xlo, 0.f));
  const int x1 = int(fminf(xhi, float(bp.tiles_x - 1)));
  y0 = int(fmaxf(ylo, 0.f));
  const int y1 = int(fminf(yhi, float(bp.tiles_y - 1)));
  nx = x1 - x0 + 1;
  return nx * (y1 - y0 + 1);
}

template <bool ANISO>
__device__ __forceinline__ int tile_rect_of(const float4* __restrict__ rec, const float4* __restrict__ shape,
                                            long long g, const BinParams& bp, int& x0, int& y0, int& nx) {
  if constexpr (ANISO) return tile_rect_aniso(rec[g], shape[g], bp, x0, y0, nx);
  else return tile_rect(rec[g], bp, x0, y0, nx);
}

// Tiles of a fill layer: the union of the bin rectangles of a block of its
// grid's Gaussians.  They share sigma and sit on a grid, so the union runs
// from the rectangle of the block's corner with the smallest x and y (r0) to
// that of the corner with the largest (r1), by the same float32 rule.
__device__ __forceinline__ int layer_rect(const float4 r0, const float4 r1, const BinParams& bp, int& x0, int& y0,
                                          int& nx) {
  const float ks = __fmul_rn(bp.k_sigma, r0.z);
  const float xlo = floorf(__fmul_rn(__fsub_rn(r0.x, ks), bp.inv_tile));
  const float xhi = floorf(__fmul_rn(__fadd_rn(r1.x, ks), bp.inv_tile));
  const float ylo = floorf(__fmul_rn(__fsub_rn(r0.y, ks), bp.inv_tile));
  const float yhi = floorf(__fmul_rn(__fadd_rn(r1.y, ks), bp.inv_tile));
  const bool ok = r0.z > 0.f && xhi >= 0.f && yhi >= 0.f && xlo <= float(bp.tiles_x - 1) &&
                  ylo <= float(bp.tiles_y - 1) && xlo <= xhi && ylo <= yhi;
  if (!ok) return 0;
  x0 = int(fmaxf(xlo, 0.f));
  const int x1 = int(fminf(xhi, float(bp.tiles_x - 1)));
  y0 = int(fmaxf(ylo, 0.f));
  const int y1 = int(fminf(yhi, float(bp.tiles_y - 1)));
  nx = x1 - x0 + 1;
  return nx * (y1 - y0 + 1);
}

// Tiles of a fill layer restricted to its live grid points: the layer rule
// above applied to the columns and rows between the live extremes (the
// x of a column is that of its record in the first row, the y of a row that
// of its first record).  Live points are the only ones per-Gaussian pairs
// would list, so nothing that composites is left out.
__device__ __forceinline__ int layer_rect_live(const float4* __restrict__ rec, const CurvePlan& p, long long G,
                                               const BinParams& bp, int c, int& x0, int& y0, int& nx) {
  const int2 lo = bp.lmin[c], hi = bp.lmax[c];
  if (hi.x < lo.x || hi.y < lo.y || lo.x < 0 || lo.y < 0 || hi.x >= p.nx || hi.y >= p.ny) return 0;
  const long long last = G - 1;
  const float4 rx0 = rec[min((long long)p.g_off + lo.x, last)], rx1 = rec[min((long long)p.g_off + hi.x, last)];
  const float4 ry0 = rec[min((long long)p.g_off + (long long)lo.y * p.nx, last)];
  const float4 ry1 = rec[min((long long)p.g_off + (long long)hi.y * p.nx, last)];
  return layer_rect(make_float4(rx0.x, ry0.y, rx0.z, rx0.w), make_float4(rx1.x, ry1.y, rx1.z, rx1.w), bp, x0, y0, nx);
}

// Tile count of Gaussian g in the pair emission, and its rectangle.  In
// fill-layer mode a fill Gaussian counts only as its layer's first one, and
// only when count_layers is set (the binning counts layers separately).
template <bool ANISO>
__device__ __forceinline__ int gaussian_tiles(const float4* __restrict__ rec, const float4* __restrict__ shape,
                                              const int* __restrict__ cflags, const CurvePlan* __restrict__ plan,
                                              long long g, int cv, int G, const BinParams& bp, bool count_layers,
                                              bool& layer, int& x0, int& y0, int& nx) {
  layer = false;
  if (cv < 0 || cv >= bp.n_curves) return 0;
  if (bp.fill_layers && (cflags[cv] & NS_FILLED)) {
    const CurvePlan& p = plan[cv];
    if (g != p.g_off || p.count <= 0) return 0;
    layer = true;
    return count_layers ? layer_rect_live(rec, p, G, bp, cv, x0, y0, nx) : 0;
  }
  return tile_rect_of<ANISO>(rec, shape, g, bp, x0, y0, nx);
}

__device__ __forceinline__ int block_excl_scan_int(int v, int* s_warp, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < nw ? s_warp[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) s_warp[lane] = t;
  }
  __syncthreads();
  total = s_warp[nw - 1];
  const int r = (w > 0 ? s_warp[w - 1] : 0) + x - v;
  __syncthreads();
  return r;
}

// The exponent coefficient -1 / (2 sigma^2) of Eq. 9.
__device__ __forceinline__ float ncoef(float sigma) { return __fdiv_rn(-0.5f, __fmul_rn(sigma, sigma)); }
// The same coefficient times log2(e), for exponentials taken as powers of 2.
__device__ __forceinline__ float ncoef2(float sigma) { return __fmul_rn(ncoef(sigma), 1.44269504088896341f); }
// 2^x by the special-function unit's approximation (relative error near 2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Squared reach of a Gaussian: beyond it alpha < alpha_min for certain
// (a margin of 1e-3 in the logarithm covers the rounding of exp and of d^2).
__device__ __forceinline__ float reach2(float sigma, float o, float log_amin) {
  if (!(log_amin > -1e30f)) return FLT_MAX;
  return 2.f * sigma * sigma * (__logf(o) - log_amin + 1e-3f);
}

// Counts tiles per Gaussian and prepares the per-Gaussian blend constants.
// Tangent-aligned Gaussians keep the exponent's conic: prep = {mu_x, mu_y, A,
// o}, prep2 = {B2, C} with exponent A dx^2 + B2 dx dy + C dy^2.
template <bool ANISO>
__global__ void __launch_bounds__(256) k_bin_count(const float4* __restrict__ rec, const float4* __restrict__ shape,
                                                   const int* __restrict__ gcurve,
                                                   const int* __restrict__ cflags, const int* __restrict__ gcount,
                                                   BinParams bp, int* bsum, DevState* st, float4* prep,
                                                   float2* prep2, float2* reach, const CurvePlan* __restrict__ plan) {
  grid_dep_wait();
  __shared__ int s_warp[32];
  const int G = min(*gcount, bp.gcap);
  // with nurbs_sample's live boxes and culled count a fill Gaussian needs
  // nothing here (its layer is counted per curve): only its curve is read
  const bool fast = sampled_boxes(bp, st);
  if (fast && blockIdx.x == 0 && threadIdx.x == 0 && G > 0 && st->culled_s) atomicAdd(&st->culled, st->culled_s);
  // persistent over the binning blocks (most of them skip at once with fill layers)
  for (int blk = blockIdx.x; (long long)blk * kBinItems < G; blk += gridDim.x) {
    const long long base = (long long)blk * kBinItems;
    // a block that holds no stroke Gaussian (nurbs_sample marked the others)
    // holds fill Gaussians only: nothing to count here
    if (fast && !bp.bmix[blk]) {
      if (threadIdx.x == 0) {
        bsum[blk] = 0;
        bp.bflag[blk] = 0;
      }
      continue;
    }
    int cnt = 0, culled = 0, other = 0;
    // the block total is all that is kept, so consecutive threads take
    // consecutive Gaussians (coalesced loads and stores)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const long long g = base + k * 256 + threadIdx.x;
      int live_key = -1, live_ix = 0, live_iy = 0;   // fill layers: live grid point of curve live_key
      bool skip = false;
      if (g < G && fast) {
        const int cv = gcurve[g];
        skip = cv >= 0 && cv < bp.n_curves && (cflags[cv] & NS_FILLED);
      }
      if (g < G && !skip) {
        other = 1;
        const float4 r = rec[g];
        int x0, y0, nx;
        const int cv = gcurve[g];
        bool layer;
        const int nt = gaussian_tiles<ANISO>(rec, shape, cflags, plan, g, cv, G, bp, false, layer, x0, y0, nx);
        cnt += nt;
        if (bp.fill_layers && cv >= 0 && cv < bp.n_curves && (cflags[cv] & NS_FILLED) && r.z > 0.f && r.w > 0.f &&
            r.w >= bp.alpha_min) {
          const CurvePlan& p = plan[cv];
          const float ih = 1.f / p.h;
          live_key = cv;
          live_ix = __float2int_rn((r.x - p.x0) * ih - 0.5f);
          live_iy = __float2int_rn((r.y - p.y0) * ih - 0.5f);
        }
        if (nt && !layer) {   // only Gaussians binned on their own are read through these
          // 1/sigma, negative for the Gaussians of filled curves (their centre and
          // sigma get no gradient through the chain, so the adjoint may skip
          // them).  The curve's flag decides: a fill point's aux can equal the
          // contour marker -1 (~0: outside, nearest segment 0).
          const float isg = 1.f / r.z;
          const float sgn_isg = (cflags[cv] & NS_FILLED) ? -isg : isg;
          if constexpr (ANISO) {
            const float4 sh = shape[g];
            const float it = 1.f / (sh.x * sh.x), in = 1.f / (r.z * r.z);
            const float A = -0.5f * (sh.y * sh.y * it + sh.z * sh.z * in);
            const float B2 = -sh.y * sh.z * (it - in);
            const float Cc = -0.5f * (sh.z * sh.z * it + sh.y * sh.y * in);
            prep[g] = make_float4(r.x, r.y, A, r.w);
            prep2[g] = make_float2(B2, Cc);
            reach[g] = make_float2(reach2(fmaxf(sh.x, r.z), r.w, bp.log_amin), sgn_isg);
          } else {
            prep[g] = make_float4(r.x, r.y, ncoef(r.z), r.w);
            reach[g] = make_float2(reach2(r.z, r.w, bp.log_amin), sgn_isg);
          }
        }
        culled += (r.z > 0.f && r.w < bp.alpha_min) ? 1 : 0;
      }
      if (bp.fill_layers && !fast) {   // warp-uniform
        // extremes of the live grid points per curve: lanes of one curve reduce, one lane adds
        const unsigned int peers = __match_any_sync(0xffffffffu, live_key);
        if (live_key >= 0) {
          const int mnx = __reduce_min_sync(peers, live_ix), mxx = __reduce_max_sync(peers, live_ix);
          const int mny = __reduce_min_sync(peers, live_iy), mxy = __reduce_max_sync(peers, live_iy);
          if ((threadIdx.x & 31) == __ffs(peers) - 1) {
            atomicMin(&bp.lmin[live_key].x, mnx);
            atomicMax(&bp.lmax[live_key].x, mxx);
            atomicMin(&bp.lmin[live_key].y, mny);
            atomicMax(&bp.lmax[live_key].y, mxy);
          }
        }
      }
    }
    int total;
    block_excl_scan_int(cnt, s_warp, total);
    int ctot;
    block_excl_scan_int(culled, s_warp, ctot);
    const int any_other = __syncthreads_or(other);
    if (threadIdx.x == 0) {
      bsum[blk] = total;
      if (bp.fill_layers) bp.bflag[blk] = fast ? any_other : 1;
      if (ctot) atomicAdd(&st->culled, (unsigned long long)ctot);
    }
  }
}

// Fill layers: each filled curve's tile count (from its live grid points)
// joins the count of the binning block that holds its first Gaussian, where
// k_bin_emit writes the layer's pairs.
__global__ void k_layer_count(ns_curves cv, const CurvePlan* __restrict__ plan, const float4* __restrict__ rec,
                              const int* __restrict__ gcount, BinParams bp, int* bsum, const DevState* st) {
  grid_dep_wait();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cv.n_curves) return;
  bp.lcount[c] = 0;
  if (!(cv.flags[c] & NS_FILLED)) return;
  const CurvePlan p = plan[c];
  const long long G = min((long long)*gcount, (long long)bp.gcap);
  if (p.g_off < 0 || p.g_off >= G || p.count <= 0) return;
  if (sampled_boxes(bp, st)) {   // the live box nurbs_sample found
    const int4 b = bp.lbox[c];
    bp.lmin[c] = make_int2(b.x, b.y);
    bp.lmax[c] = make_int2(b.z, b.w);
  }
  int x0, y0, nx;
  const int nt = layer_rect_live(rec, p, G, bp, c, x0, y0, nx);
  bp.lcount[c] = nt;
  if (nt) atomicAdd(&bsum[p.g_off / kBinItems], nt);
}

// The pairs of the fill layers whose first Gaussian lies in a binning block of
// fill Gaussians only (k_bin_emit leaves those blocks out), one block per
// curve, a pair per thread: after the pairs of the layers that start earlier
// in the same binning block (the curves before it in front-to-back order), in
// the pair order k_bin_emit would give them.
__global__ void __launch_bounds__(128) k_layer_emit(ns_curves cv, const CurvePlan* __restrict__ plan,
                                                    const float4* __restrict__ rec, const int* __restrict__ gcount,
                                                    const int* __restrict__ curve_scene, BinParams bp,
                                                    const int* __restrict__ boff, const int* __restrict__ order,
                                                    uint32_t* keys, uint32_t* vals, long long pcap,
                                                    const DevState* st) {
  grid_dep_wait();
  const int c = blockIdx.x;
  if (c >= cv.n_curves || !sampled_boxes(bp, st)) return;
  const int nt = bp.lcount[c];
  if (nt <= 0) return;
  const CurvePlan p = plan[c];
  const long long G = min((long long)*gcount, (long long)bp.gcap);
  const int blk = p.g_off / kBinItems;
  if (bp.bflag[blk]) return;   // a mixed block: k_bin_emit writes this layer's pairs
  // position in front-to-back order: within its scene the last curve comes first
  int s0 = 0, s1 = cv.n_curves;
  if (cv.scene_curve_offset) {
    s0 = cv.scene_curve_offset[p.scene];
    s1 = cv.scene_curve_offset[p.scene + 1];
  }
  long long off = boff[blk];
  const long long base = (long long)blk * kBinItems;
  for (int q = s0 + (s1 - 1 - c) - 1; q >= 0; --q) {
    const int c2 = order[q];
    if (plan[c2].g_off < base) break;
    off += bp.lcount[c2];
  }
  int x0, y0, nx;
  layer_rect_live(rec, p, G, bp, c, x0, y0, nx);
  const int sbase = curve_scene[c] * bp.tiles_per_scene;
  const uint32_t val = uint32_t(p.g_off) | kLayerBit;
  for (int j = threadIdx.x; j < nt && off + j < pcap; j += blockDim.x) {
    const int jy = j / nx;
    keys[off + j] = uint32_t(sbase + (y0 + jy) * bp.tiles_x + x0 + (j - jy * nx));
    vals[off + j] = val;
  }
}

__global__ void k_scan_small(int* vals, const int* gcount, int gcap, int items_per_block, DevState* st,
                             long long cap, uint32_t* zero, int nzero) {
  grid_dep_wait();
  for (int i = threadIdx.x; i < nzero; i += blockDim.x) zero[i] = 0u;   // the radix sort's digit totals
  const int G = min(*gcount, gcap);
  const int n = (G + items_per_block - 1) / items_per_block;
  long long t1[1];
  block_scan_multi<1>(
      n, [&](int i, long long v[1]) { v[0] = vals[i]; },
      [&](int i, const long long off[1]) { vals[i] = int(off[0] < 0x7fffffffLL ? off[0] : 0x7fffffffLL); }, t1);
  if (threadIdx.x == 0) {
    const long long tot = t1[0];
    st->pair_total = (unsigned long long)tot;
    st->pair_count = int(tot < cap ? tot : cap);
    if (tot > cap) raise_status(st, NS_ERR_CAPACITY);
  }
}

template <bool ANISO>
__global__ void __launch_bounds__(256) k_bin_emit(const float4* __restrict__ rec, const float4* __restrict__ shape,
                                                  const int* __restrict__ gcurve,
                                                  const int* __restrict__ gcount, const int* __restrict__ curve_scene,
                                                  BinParams bp, const int* __restrict__ boff, uint32_t* keys,
                                                  uint32_t* vals, long long pcap, const int* __restrict__ cflags,
                                                  const CurvePlan* __restrict__ plan) {
  grid_dep_wait();
  __shared__ int s_warp[32];
  __shared__ int s_off[kBinItems];    // tile count, then exclusive offset in Gaussian order
  __shared__ int2 s_rect[kBinItems];  // {x0 | nx << 16, y0 | ny << 16}
  const int G = min(*gcount, bp.gcap);
  // persistent over the binning blocks (most of them skip at once with fill layers)
  for (int blk = blockIdx.x; (long long)blk * kBinItems < G; blk += gridDim.x) {
    const long long base = (long long)blk * kBinItems;
    // a block whose Gaussians emit no pair (the inside of a fill layer, culled
    // points) has the same offset as the next block
    if (base + kBinItems < G && boff[blk + 1] == boff[blk]) continue;
    // a block of fill Gaussians only, with nurbs_sample's live boxes: its layers'
    // pairs come from k_layer_emit
    if (bp.fill_layers && !bp.bflag[blk]) continue;
    __syncthreads();   // the previous block's pairs have read s_off and s_rect
    // 1. rectangles, consecutive threads on consecutive Gaussians (coalesced)
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int gl = k * 256 + threadIdx.x;
      const long long g = base + gl;
      int c = 0, x0 = 0, y0 = 0, nx = 1;
      if (g < G) {
        bool layer;
        c = gaussian_tiles<ANISO>(rec, shape, cflags, plan, g, gcurve[g], G, bp, true, layer, x0, y0, nx);
      }
      s_off[gl] = c;
      s_rect[gl] = make_int2(x0 | (nx << 16), y0 | ((c ? c / nx : 0) << 16));
    }
    __syncthreads();
    // 2. exclusive offsets in Gaussian order (each thread 8 consecutive)
    int cnt[8], tot = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      cnt[k] = s_off[threadIdx.x * 8 + k];
      tot += cnt[k];
    }
    int btot;
    int run = block_excl_scan_int(tot, s_warp, btot);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      s_off[threadIdx.x * 8 + k] = run;
      run += cnt[k];
    }
    __syncthreads();
    // 3. pairs, consecutive threads on consecutive Gaussians again
    const long long boff0 = boff[blk];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int gl = k * 256 + threadIdx.x;
      const long long g = base + gl;
      if (g >= G) continue;
      const int2 rr = s_rect[gl];
      const int nx = rr.x >> 16, ny = rr.y >> 16;
      const int c = nx * ny;
      if (!c) continue;
      const int x0 = rr.x & 0xffff, y0 = rr.y & 0xffff;
      const int cv = gcurve[g];
      const int sbase = curve_scene[cv] * bp.tiles_per_scene;
      const uint32_t val = uint32_t(g) | ((bp.fill_layers && (cflags[cv] & NS_FILLED)) ? kLayerBit : 0u);
      long long off = boff0 + s_off[gl];
      for (int j = 0; j < c; ++j, ++off) {
        if (off >= pcap) break;
        const int tx = x0 + j % nx;
        const int ty = y0 + j / nx;
        keys[off] = uint32_t(sbase + ty * bp.tiles_x + tx);
        vals[off] = val;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (tile, Gaussian) pairs on the tile bits

// Per sort block, the count of each digit (digit-major: hist[digit][block]);
// the digit totals over all blocks are added to totals[digit] (zeroed by
// k_scan_small).
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys, const DevState* st,
                                                             int shift, int bits, uint32_t* hist, uint32_t* totals) {
  grid_dep_wait();
  constexpr int kPer = kSortItems / kSortThreads;
  __shared__ uint32_t h[256];
  const int n = st->pair_count;
  const int nb = (n + kSortItems - 1) / kSortItems;
  const int nd = 1 << bits;
  // sort blocks of kSortItems pairs, grid-stride (the grid is sized by the
  // capacity, the pairs are known on the device only)
  for (int vb = blockIdx.x; vb < nb; vb += gridDim.x) {
    for (int d = threadIdx.x; d < nd; d += kSortThreads) h[d] = 0;
    const long long base = (long long)vb * kSortItems + threadIdx.x;
    uint32_t kk[kPer];   // every load in flight before the first count
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const long long i = base + r * kSortThreads;
      kk[r] = i < n ? keys[i] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPer; ++r)
      if (base + r * kSortThreads < n) atomicAdd(&h[(kk[r] >> shift) & (nd - 1)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += kSortThreads) {
      const uint32_t c = h[d];
      hist[(long long)d * nb + vb] = c;
      if (c) atomicAdd(&totals[d], c);
    }
    __syncthreads();
  }
}

// Exclusive scan of the digit-major histogram hist[digit][block]: one block
// per digit scans its row, starting from the total of all smaller digits
// (totals, from k_radix_hist).
__device__ __forceinline__ uint32_t block_sum_u32(uint32_t v, uint32_t* s_warp) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
  __syncthreads();
  uint32_t t = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_warp[w];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(256) k_radix_scan(uint32_t* hist, const DevState* st,
                                                    const uint32_t* __restrict__ totals) {
  grid_dep_wait();
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_carry;
  const int nb = (st->pair_count + kSortItems - 1) / kSortItems;
  uint32_t base = 0;
  for (int d = threadIdx.x; d < (int)blockIdx.x; d += blockDim.x) base += totals[d];
  base = block_sum_u32(base, s_warp);
  if (threadIdx.x == 0) s_carry = base;
  __syncthreads();
  uint32_t* row = hist + (long long)blockIdx.x * nb;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
    const int i = b0 + threadIdx.x;
    const uint32_t v = i < nb ? row[i] : 0u;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
      uint32_t t = lane < nw ? s_warp[lane] : 0u;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < nw) s_warp[lane] = t;
    }
    __syncthreads();
    const uint32_t excl = s_carry + (w > 0 ? s_warp[w - 1] : 0u) + x - v;
    if (i < nb) row[i] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry = excl + v;
    __syncthreads();
  }
}

// Each warp ranks its 512 consecutive pairs in 16 rounds of 32 with
// __match_any_sync; per-warp digit counters keep the order stable.
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                       const uint32_t* __restrict__ vin, uint32_t* kout,
                                                       uint32_t* vout, const uint32_t* __restrict__ hist,
                                                       const DevState* st, int shift, int bits) {
  grid_dep_wait();
  constexpr int kWarps = kSortThreads / 32, kPerWarp = kSortItems / kWarps, kRounds = kPerWarp / 32;
  __shared__ uint32_t wcnt[kWarps][256];
  __shared__ uint32_t dstart[256];        // first position of each digit in the block's sorted order
  __shared__ uint32_t gbase[256];         // global position of each digit's first item of this block
  __shared__ uint32_t s_key[kSortItems];  // the block's items in digit order (stable)
  __shared__ uint32_t s_val[kSortItems];
  const int n = st->pair_count;
  const int nb = (n + kSortItems - 1) / kSortItems;
  const int nd = 1 << bits;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // sort blocks of kSortItems pairs, grid-stride (see k_radix_hist)
  for (int vb = blockIdx.x; vb < nb; vb += gridDim.x) {
    __syncthreads();   // the previous block's shared arrays are read
    for (int d = lane; d < nd; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    const long long blk0 = (long long)vb * kSortItems;
    const int nblk = (int)min((long long)kSortItems, n - blk0);
    const long long base = blk0 + (long long)w * kPerWarp;
    uint32_t key[kRounds], val[kRounds];
    uint32_t rank[kRounds];
    // every load in flight first: the rounds below are separated by
    // __syncwarp, which would hold each round's loads back until the last
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const long long i = base + r * 32 + lane;
      const bool ok = i < n;
      key[r] = ok ? kin[i] : 0u;
      val[r] = ok ? vin[i] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const long long i = base + r * 32 + lane;
      const bool ok = i < n;
      const uint32_t d = ok ? (key[r] >> shift) & (nd - 1) : 0xffffffffu;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t below = peers & ((1u << lane) - 1u);
      const uint32_t base_cnt = ok ? wcnt[w][d] : 0u;
      rank[r] = base_cnt + __popc(below);
      __syncwarp();
      if (ok && below == 0u) wcnt[w][d] = base_cnt + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per digit: offsets of the warps inside the block's digit run, the run's
    // start in the block's sorted order, and its global position
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {
      uint32_t acc = 0;
#pragma unroll
      for (int ww = 0; ww < kWarps; ++ww) {
        const uint32_t c = wcnt[ww][d];
        wcnt[ww][d] = acc;
        acc += c;
      }
      dstart[d] = acc;   // the digit's count for now
      gbase[d] = hist[(long long)d * nb + vb];
    }
    __syncthreads();
    if (threadIdx.x < 32) {   // exclusive scan of the digit counts (nd <= 256)
      uint32_t run = 0;
      for (int c0 = 0; c0 < nd; c0 += 32) {
        const int d = c0 + lane;
        uint32_t v = d < nd ? dstart[d] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        if (d < nd) dstart[d] = run + x - v;
        run += __shfl_sync(0xffffffffu, x, 31);
      }
    }
    __syncthreads();
    // stable local placement in shared memory
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const long long i = base + r * 32 + lane;
      if (i < n) {
        const uint32_t d = (key[r] >> shift) & (nd - 1);
        const uint32_t pos = dstart[d] + wcnt[w][d] + rank[r];
        s_key[pos] = key[r];
        s_val[pos] = val[r];
      }
    }
    __syncthreads();
    // contiguous runs per digit: consecutive threads write consecutive positions
    for (int j = threadIdx.x; j < nblk; j += blockDim.x) {
      const uint32_t k = s_key[j];
      const uint32_t d = (k >> shift) & (nd - 1);
      const uint32_t pos = gbase[d] + (uint32_t(j) - dstart[d]);
      kout[pos] = k;
      vout[pos] = s_val[j];
    }
  }
}
__global__ void k_ranges(const uint32_t* __restrict__ keys, const DevState* st, int2* ranges) {
  grid_dep_wait();
  const int n = st->pair_count;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = int(i);
    if (i == n - 1 || keys[i + 1] != t) ranges[t].y = int(i + 1);
  }
}

// ---------------------------------------------------------------------------
// compositing
//
// Thread layout: one TILE x TILE tile per block.  A warp owns an 8-wide,
// (4 PPT)-tall sub-block; lane l handles the PPT pixels (l & 7, (l >> 3) + 4k),
// k < PPT.  Each warp streams its tile's list on its own, 32 entries at a
// time, staged in the warp's slice of shared memory (no block barriers, so a
// warp whose pixels are all done leaves at once).  Before the warp evaluates a
// Gaussian it tests, one Gaussian per lane and a ballot, whether the Gaussian
// can reach alpha_min anywhere in its sub-block: alpha >= alpha_min needs
// d^2 <= 2 sigma^2 ln(o / alpha_min); the test uses the sub-block's nearest
// point with a margin of 1e-3 in the logarithm, so a Gaussian it rejects would
// have been skipped by the alpha < alpha_min rule at every pixel of the
// sub-block.  The result is the same as evaluating every pair; only the work
// changes.  With alpha_min = 0 nothing is rejected.  TILE and PPT change only
// the work decomposition, never the result: every pixel still walks its
// tile's list in order.
//
// Per-Gaussian constants are prepared once by k_bin_count:
//   prep  = {mu_x, mu_y, ncoef = -1/(2 sigma^2), o}
//   reach = {squared reach, 1/sigma, negative for fill Gaussians}

struct BlendParams {
  float alpha_min, alpha_max, t_min;
  float bg0, bg1, bg2;
  int W, H, tiles_x, tiles_per_scene;
};

// alpha = min(alpha_max, o exp(ncoef d^2)) (Eq. 9), written with explicit
// roundings so that the forward and the backward kernels compute the same bits.
__device__ __forceinline__ float gauss_alpha(float fx, float fy, float4 q, float amax, float& dx, float& dy,
                                             float& d2, float& e) {
  dx = __fsub_rn(fx, q.x);
  dy = __fsub_rn(fy, q.y);
  d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
  e = __expf(__fmul_rn(q.z, d2));
  return fminf(__fmul_rn(q.w, e), amax);
}

// Alpha of a tangent-aligned Gaussian from its conic (prep {mu_x, mu_y, A, o},
// q2 = {B2, C}): exponent A dx^2 + B2 dx dy + C dy^2, the same roundings in the
// forward and the backward kernels.
__device__ __forceinline__ float gauss_alpha_aniso(float fx, float fy, float4 q, float2 q2, float amax, float& dx,
                                                   float& dy, float& e) {
  dx = __fsub_rn(fx, q.x);
  dy = __fsub_rn(fy, q.y);
  const float E = __fmaf_rn(q.z, __fmul_rn(dx, dx), __fmaf_rn(q2.x, __fmul_rn(dx, dy), __fmul_rn(q2.y, __fmul_rn(dy, dy))));
  e = __expf(E);
  return fminf(__fmul_rn(q.w, e), amax);
}

// Squared distance from (x, y) to the rectangle [x0, x1] x [y0, y1].
__device__ __forceinline__ float rect_d2(float x, float y, float x0, float x1, float y0, float y1) {
  const float dx = fmaxf(fmaxf(x0 - x, x - x1), 0.f);
  const float dy = fmaxf(fmaxf(y0 - y, y - y1), 0.f);
  return dx * dx + dy * dy;
}

// Adds a per-thread count to a device counter, one atomic per warp.
__device__ __forceinline__ void count_evals(unsigned long long* ctr, unsigned int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(ctr, (unsigned long long)v);
}

template <int TILE, int PPT>
struct BlendGeom {
  static constexpr int kWarpsX = TILE / 8;
  static constexpr int kWarpsY = TILE / (4 * PPT);
  static constexpr int kWarps = kWarpsX * kWarpsY;
  static constexpr int kThreads = 32 * kWarps;
  static constexpr int kMinBlocks = 1024 / kThreads;   // 1024 resident threads: up to 64 registers each
  // the adjoint with 4 pixels per thread keeps 4 x 8 floats of pixel state: allow 128 registers
  static constexpr int kMinBlocksBwd = (PPT == 4 ? 512 : 1024) / kThreads > 0 ? (PPT == 4 ? 512 : 1024) / kThreads : 1;
  static_assert(kWarpsY >= 1 && TILE % (4 * PPT) == 0, "sub-block taller than the tile");
};

// Scene, pixel column and first row of this lane, and the warp's rectangle.
template <int TILE, int PPT>
__device__ __forceinline__ void tile_pixels(const BlendParams& bp, int& s, int& px, int& py0, float4& rect) {
  using Gm = BlendGeom<TILE, PPT>;
  const int tile = blockIdx.x;
  s = tile / bp.tiles_per_scene;
  const int t = tile - s * bp.tiles_per_scene;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx = (t % bp.tiles_x) * TILE + (w % Gm::kWarpsX) * 8;
  const int by = (t / bp.tiles_x) * TILE + (w / Gm::kWarpsX) * 4 * PPT;
  px = bx + (lane & 7);
  py0 = by + (lane >> 3);
  rect = make_float4(bx + 0.5f, bx + 7.5f, by + 0.5f, by + 4.f * PPT - 0.5f);
}

template <int TILE, int PPT, int C, bool ANISO>
__global__ void __launch_bounds__(BlendGeom<TILE, PPT>::kThreads, BlendGeom<TILE, PPT>::kMinBlocks)
    k_blend_fwd(const int2* __restrict__ ranges, const uint32_t* __restrict__ gid, const float4* __restrict__ prep,
                const float2* __restrict__ prep2, const float2* __restrict__ reach, const int* __restrict__ gcurve,
                const float4* __restrict__ color, BlendParams bp, float* image, float* Tfinal, int* nlast,
                DevState* st) {
  grid_dep_wait();
  using Gm = BlendGeom<TILE, PPT>;
  __shared__ float4 s_q[Gm::kWarps][32];
  __shared__ float4 s_c[Gm::kWarps][32];
  __shared__ float2 s_q2[ANISO ? Gm::kWarps : 1][32];
  int s, px, py0;
  float4 wr;
  tile_pixels<TILE, PPT>(bp, s, px, py0, wr);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float fx = px + 0.5f;
  const int2 rg = ranges[blockIdx.x];
  const int n = rg.y - rg.x;
  float T[PPT], acc[PPT][C];
  bool done[PPT];
  int last[PPT], stop[PPT];   // stop: entries walked up to the one that ended the pixel (0 = not ended)
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    T[k] = 1.f;
    done[k] = !(px < bp.W && py0 + 4 * k < bp.H);
    last[k] = 0;
    stop[k] = 0;
#pragma unroll
    for (int ch = 0; ch < C; ++ch) acc[k][ch] = 0.f;
  }
  auto all_done = [&]() {
    bool d = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) d = d && done[k];
    return d;
  };
  unsigned int evals = 0, contribs = 0;
  for (int base = 0; base < n && !__all_sync(0xffffffffu, all_done()); base += 32) {
    const int j = base + lane;
    bool hit = false;
    const uint32_t g = j < n ? gid[rg.x + j] : kLayerBit;
    if (!(g & kLayerBit)) {   // fill-layer entries (settings of another pass) are never read here
      const float4 q = prep[g];
      hit = rect_d2(q.x, q.y, wr.x, wr.y, wr.z, wr.w) <= reach[g].x;
      if (hit) {
        s_q[w][lane] = q;
        s_c[w][lane] = color[gcurve[g]];
        if (ANISO) s_q2[ANISO ? w : 0][lane] = prep2[g];
      }
    }
    unsigned int mask = __ballot_sync(0xffffffffu, hit);
    __syncwarp();
    while (mask) {
      const int b = __ffs(mask) - 1;
      mask &= mask - 1;
      const float4 q = s_q[w][b];
      const float2 q2 = ANISO ? s_q2[ANISO ? w : 0][b] : make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (done[k]) continue;
        ++evals;
        float dx, dy, d2, e;
        const float a = ANISO ? gauss_alpha_aniso(fx, py0 + 4 * k + 0.5f, q, q2, bp.alpha_max, dx, dy, e)
                              : gauss_alpha(fx, py0 + 4 * k + 0.5f, q, bp.alpha_max, dx, dy, d2, e);
        if (a < bp.alpha_min) continue;
        const float test = T[k] * (1.f - a);
        if (test < bp.t_min) {
          done[k] = true;
          stop[k] = base + b + 1;
          continue;
        }
        const float wgt = a * T[k];
        const float4 cc = s_c[w][b];
        acc[k][0] = fmaf(cc.x, wgt, acc[k][0]);
        if (C == 3) {
          acc[k][1] = fmaf(cc.y, wgt, acc[k][1]);
          acc[k][2] = fmaf(cc.z, wgt, acc[k][2]);
        }
        T[k] = test;
        last[k] = base + b + 1;
        ++contribs;
      }
    }
    __syncwarp();
  }
  count_evals(&st->blend_evals, evals);
  count_evals(&st->blend_contribs, contribs);
  unsigned int visits = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k)
    if (px < bp.W && py0 + 4 * k < bp.H) visits += stop[k] ? stop[k] : n;
  count_evals(&st->blend_visits, visits);
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int py = py0 + 4 * k;
    if (px < bp.W && py < bp.H) {
      const long long pix = ((long long)s * bp.H + py) * bp.W + px;
      float* out = image + pix * C;
      out[0] = acc[k][0] + T[k] * bp.bg0;
      if (C == 3) {
        out[1] = acc[k][1] + T[k] * bp.bg1;
        out[2] = acc[k][2] + T[k] * bp.bg2;
      }
      Tfinal[pix] = T[k];
      nlast[pix] = last[k];
    }
  }
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
               : "memory");
}

// Rows of the per-Gaussian gradients: {dmu_x, dmu_y, dsigma, 0, do, dr, dg, db};
// tangent-aligned: {dmu_x, dmu_y, dA, dB2, do, dr, dg, db, dC, 0, 0, 0} (the
// conic of gauss_alpha_aniso).
template <bool ANISO>
struct GradRow {
  static constexpr int kFloats = ANISO ? 12 : 8;
};

template <int TILE, int PPT, int C, bool ANISO>
__global__ void __launch_bounds__(BlendGeom<TILE, PPT>::kThreads, BlendGeom<TILE, PPT>::kMinBlocksBwd)
    k_blend_bwd(const int2* __restrict__ ranges, const uint32_t* __restrict__ gid, const float4* __restrict__ prep,
                const float2* __restrict__ prep2, const float2* __restrict__ reach, const int* __restrict__ gcurve,
                const float4* __restrict__ color, BlendParams bp, const float* __restrict__ dimage,
                const float* __restrict__ Tfinal, const int* __restrict__ nlast, float* dgauss, DevState* st,
                int full_grads, float* /* per-curve colour gradients: unused, the rows carry them */) {
  grid_dep_wait();
  using Gm = BlendGeom<TILE, PPT>;
  constexpr int kRow = GradRow<ANISO>::kFloats;
  __shared__ float4 s_q[Gm::kWarps][32];
  __shared__ float4 s_c[Gm::kWarps][32];
  __shared__ float s_isig[Gm::kWarps][32];
  __shared__ uint32_t s_id[Gm::kWarps][32];
  __shared__ float2 s_q2[ANISO ? Gm::kWarps : 1][32];
  int s, px, py0;
  float4 wr;
  tile_pixels<TILE, PPT>(bp, s, px, py0, wr);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float fx = px + 0.5f;
  const int2 rg = ranges[blockIdx.x];
  float T[PPT], dI[PPT][3], Bk[PPT][3];
  int last[PPT];
  int wmax = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int py = py0 + 4 * k;
    T[k] = 1.f;
    last[k] = 0;
    Bk[k][0] = bp.bg0;
    Bk[k][1] = bp.bg1;
    Bk[k][2] = bp.bg2;
    dI[k][0] = dI[k][1] = dI[k][2] = 0.f;
    if (px < bp.W && py < bp.H) {
      const long long pix = ((long long)s * bp.H + py) * bp.W + px;
      T[k] = Tfinal[pix];
      last[k] = nlast[pix];
#pragma unroll
      for (int ch = 0; ch < C; ++ch) dI[k][ch] = dimage[pix * C + ch];
    }
    wmax = max(wmax, last[k]);
  }
  for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  unsigned int evals = 0;
  for (int base = ((wmax - 1) >> 5) << 5; base >= 0 && wmax > 0; base -= 32) {
    const int j = base + lane;
    bool hit = false;
    const uint32_t g = j < wmax ? gid[rg.x + j] : kLayerBit;
    if (!(g & kLayerBit)) {   // fill-layer entries (settings of another pass) are never read here
      const float4 q = prep[g];
      const float2 rs = reach[g];
      hit = rect_d2(q.x, q.y, wr.x, wr.y, wr.z, wr.w) <= rs.x;
      if (hit) {
        s_q[w][lane] = q;
        s_c[w][lane] = color[gcurve[g]];
        s_isig[w][lane] = rs.y;
        s_id[w][lane] = g;
        if (ANISO) s_q2[ANISO ? w : 0][lane] = prep2[g];
      }
    }
    unsigned int mask = __ballot_sync(0xffffffffu, hit);
    __syncwarp();
    while (mask) {
      const int b = 31 - __clz(mask);
      mask &= ~(1u << b);
      const float4 q = s_q[w][b];
      const float2 q2 = ANISO ? s_q2[ANISO ? w : 0][b] : make_float2(0.f, 0.f);
      const float isg_raw = s_isig[w][b];
      // fill Gaussians (negative 1/sigma) need only the opacity and colour
      // gradients unless the caller asked for every per-Gaussian gradient
      const bool geo = full_grads || isg_raw > 0.f;
      const float isg = fabsf(isg_raw);
      float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      float vC = 0.f;   // dC of a tangent-aligned Gaussian
      bool contrib = false;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (base + b >= last[k]) continue;
        ++evals;
        float dx, dy, d2 = 0.f, e;
        const float a = ANISO ? gauss_alpha_aniso(fx, py0 + 4 * k + 0.5f, q, q2, bp.alpha_max, dx, dy, e)
                              : gauss_alpha(fx, py0 + 4 * k + 0.5f, q, bp.alpha_max, dx, dy, d2, e);
        if (a < bp.alpha_min) continue;
        contrib = true;
        T[k] = __fdividef(T[k], 1.f - a);   // transmittance in front of this Gaussian
        const float wgt = a * T[k];
        const float4 cc = s_c[w][b];
        float da = (cc.x - Bk[k][0]) * dI[k][0];
        v[5] += wgt * dI[k][0];
        Bk[k][0] = a * cc.x + (1.f - a) * Bk[k][0];
        if (C == 3) {
          da += (cc.y - Bk[k][1]) * dI[k][1] + (cc.z - Bk[k][2]) * dI[k][2];
          v[6] += wgt * dI[k][1];
          v[7] += wgt * dI[k][2];
          Bk[k][1] = a * cc.y + (1.f - a) * Bk[k][1];
          Bk[k][2] = a * cc.z + (1.f - a) * Bk[k][2];
        }
        da *= T[k];
        if (__fmul_rn(q.w, e) < bp.alpha_max) {
          v[4] += e * da;
          if (geo) {
            if (ANISO) {
              // dalpha/dE = alpha; dE/dmu = -(2A dx + B2 dy, B2 dx + 2C dy), dE/d{A, B2, C} = {dx^2, dx dy, dy^2}
              const float ga = da * a;
              v[0] -= ga * (2.f * q.z * dx + q2.x * dy);
              v[1] -= ga * (q2.x * dx + 2.f * q2.y * dy);
              v[2] += ga * dx * dx;
              v[3] += ga * dx * dy;
              vC += ga * dy * dy;
            } else {
              const float aa = da * a * isg * isg;   // dalpha/dmu = alpha (x - mu) / sigma^2
              v[0] += aa * dx;
              v[1] += aa * dy;
              v[2] += aa * d2 * isg;                  // dalpha/dsigma = alpha d^2 / sigma^3
            }
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
        if (geo) {
          // value k of the warp total sits in lane 4k; gather 0..3 into lane 0
          // and 4..7 into lane 16, one 16-byte vector reduction each
          const float t = warp_sum8(v);
          const float t1 = __shfl_down_sync(0xffffffffu, t, 4);
          const float t2 = __shfl_down_sync(0xffffffffu, t, 8);
          const float t3 = __shfl_down_sync(0xffffffffu, t, 12);
          if ((lane & 15) == 0) {
            float* d = dgauss + (long long)s_id[w][b] * kRow + (lane >> 2);
            red_add_v4(d, t, t1, t2, t3);
          }
          if (ANISO) {
            float tc = vC;
            for (int o = 16; o > 0; o >>= 1) tc += __shfl_xor_sync(0xffffffffu, tc, o);
            if (lane == 0 && tc != 0.f) atomicAdd(dgauss + (long long)s_id[w][b] * kRow + 8, tc);
          }
        } else {
          // only {do, dr, dg, db}: value k of the warp total sits in lane 8k
          const float t = warp_sum4(v + 4);
          const float t1 = __shfl_down_sync(0xffffffffu, t, 8);
          const float t2 = __shfl_down_sync(0xffffffffu, t, 16);
          const float t3 = __shfl_down_sync(0xffffffffu, t, 24);
          if (lane == 0) red_add_v4(dgauss + (long long)s_id[w][b] * kRow + 4, t, t1, t2, t3);
        }
      }
    }
    __syncwarp();
  }
  count_evals(&st->blend_bwd_evals, evals);
  unsigned int visits = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) visits += last[k];
  count_evals(&st->blend_bwd_visits, visits);
}

// ---------------------------------------------------------------------------
// Lane-group decomposition.  A fill Gaussian's reach (about 2.5 px at h = 1)
// covers only a few of the columns of a warp's 8 x 4 PPT sub-block, so most
// lanes idle while the warp walks a Gaussian.  Here the warp splits into four
// groups of eight lanes, group g owning pixel columns 2g and 2g + 1 of the
// sub-block (all its rows), and each group walks its own list: the batch's
// Gaussians that can reach one of its pixels.  In one iteration the four
// groups work on up to four different Gaussians.  Every pixel still visits
// the Gaussians of its tile's list in list order (the groups differ only in
// which entries they skip as out of reach), so the image is bit-identical to
// the whole-warp kernels'; only the order of the gradient atomics changes.

constexpr int kLaneGroups = 4;

// Pixel of this lane in the lane-group layout: lane = 8 g + i, column
// 2 g + (i & 1), row i >> 1 (+ 4 k for the k-th pixel of the thread).
template <int TILE, int PPT>
__device__ __forceinline__ void group_pixels(const BlendParams& bp, int& s, int& px, int& py0, float& bxf,
                                             float& y0, float& y1) {
  using Gm = BlendGeom<TILE, PPT>;
  const int tile = blockIdx.x;
  s = tile / bp.tiles_per_scene;
  const int t = tile - s * bp.tiles_per_scene;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bx = (t % bp.tiles_x) * TILE + (w % Gm::kWarpsX) * 8;
  const int by = (t / bp.tiles_x) * TILE + (w / Gm::kWarpsX) * 4 * PPT;
  px = bx + 2 * (lane >> 3) + (lane & 1);
  py0 = by + ((lane >> 1) & 3);
  bxf = bx + 0.5f;
  y0 = by + 0.5f;
  y1 = by + 4.f * PPT - 0.5f;
}

// Hit masks of the four groups for the Gaussian this lane loaded (q, squared
// reach r2; valid = false for lanes past the list), and the mask of this
// lane's own group.  Group g tests the rectangle of its pixel centres
// [bxf + 2g, bxf + 2g + 1] x [y0, y1] with the same rule as the whole-warp
// kernels.
__device__ __forceinline__ unsigned int group_masks(bool valid, float qx, float qy, float r2, float bxf, float y0,
                                                    float y1, bool& any_hit) {
  const int lane = threadIdx.x & 31;
  unsigned int mine = 0;
  any_hit = false;
#pragma unroll
  for (int g = 0; g < kLaneGroups; ++g) {
    const float x0 = bxf + 2.f * g;
    const bool h = valid && rect_d2(qx, qy, x0, x0 + 1.f, y0, y1) <= r2;
    any_hit = any_hit || h;
    const unsigned int m = __ballot_sync(0xffffffffu, h);
    if ((lane >> 3) == g) mine = m;
  }
  return mine;
}

// Sum of 8 values over each aligned group of 8 lanes: lane i of the group
// receives the group total of value i (7 shuffles).
__device__ __forceinline__ float group_sum8(const float v[8]) {
  const int i = threadIdx.x & 7;
  const bool h4 = i & 4, h2 = i & 2, h1 = i & 1;
  float b[4], c[2];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float send = h4 ? v[k] : v[k + 4];
    const float keep = h4 ? v[k + 4] : v[k];
    b[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = h2 ? b[k] : b[k + 2];
    const float keep = h2 ? b[k + 2] : b[k];
    c[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  return (h1 ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, h1 ? c[0] : c[1], 1);
}

// Sum of 4 values over each aligned group of 8 lanes: lanes 0, 2, 4, 6 of the
// group receive the totals of values 0, 1, 2, 3 (4 shuffles).
__device__ __forceinline__ float group_sum4(const float v[4]) {
  const int i = threadIdx.x & 7;
  const bool h4 = i & 4, h2 = i & 2;
  float b[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float send = h4 ? v[k] : v[k + 2];
    const float keep = h4 ? v[k + 2] : v[k];
    b[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  float d = (h2 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, h2 ? b[0] : b[1], 2);
  return d + __shfl_xor_sync(0xffffffffu, d, 1);
}

template <int TILE, int PPT, int C, bool ANISO>
__global__ void __launch_bounds__(BlendGeom<TILE, PPT>::kThreads, BlendGeom<TILE, PPT>::kMinBlocks)
    k_blend_fwd_groups(const int2* __restrict__ ranges, const uint32_t* __restrict__ gid,
                       const float4* __restrict__ prep, const float2* __restrict__ prep2,
                       const float2* __restrict__ reach, const int* __restrict__ gcurve,
                       const float4* __restrict__ color, BlendParams bp, float* image, float* Tfinal, int* nlast,
                       DevState* st) {
  grid_dep_wait();
  using Gm = BlendGeom<TILE, PPT>;
  __shared__ float4 s_q[Gm::kWarps][32];
  __shared__ float4 s_c[Gm::kWarps][32];
  __shared__ float2 s_q2[ANISO ? Gm::kWarps : 1][32];
  int s, px, py0;
  float bxf, y0, y1;
  group_pixels<TILE, PPT>(bp, s, px, py0, bxf, y0, y1);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float fx = px + 0.5f;
  const int2 rg = ranges[blockIdx.x];
  const int n = rg.y - rg.x;
  float T[PPT], acc[PPT][C];
  bool done[PPT];
  int last[PPT], stop[PPT];   // stop: entries walked up to the one that ended the pixel (0 = not ended)
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    T[k] = 1.f;
    done[k] = !(px < bp.W && py0 + 4 * k < bp.H);
    last[k] = 0;
    stop[k] = 0;
#pragma unroll
    for (int ch = 0; ch < C; ++ch) acc[k][ch] = 0.f;
  }
  auto all_done = [&]() {
    bool d = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) d = d && done[k];
    return d;
  };
  unsigned int evals = 0, contribs = 0;
  for (int base = 0; base < n && !__all_sync(0xffffffffu, all_done()); base += 32) {
    const int j = base + lane;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    float r2 = -1.f;
    uint32_t g = 0;
    if (j < n) {
      g = gid[rg.x + j];
      if (!(g & kLayerBit)) {   // fill-layer entries (settings of another pass) are never read here
        q = prep[g];
        r2 = reach[g].x;
      }
    }
    bool hit;
    unsigned int m = group_masks(j < n, q.x, q.y, r2, bxf, y0, y1, hit);
    if (hit) {
      s_q[w][lane] = q;
      s_c[w][lane] = color[gcurve[g]];
      if (ANISO) s_q2[ANISO ? w : 0][lane] = prep2[g];
    }
    if (all_done()) m = 0;
    __syncwarp();
    // the non-finished lanes of a group pop the same entries in the same order
    while (__any_sync(0xffffffffu, m != 0)) {
      if (m == 0) continue;   // back to the vote: every lane votes once per iteration
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const float4 qb = s_q[w][b];
      const float2 q2 = ANISO ? s_q2[ANISO ? w : 0][b] : make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (done[k]) continue;
        ++evals;
        float dx, dy, d2, e;
        const float a = ANISO ? gauss_alpha_aniso(fx, py0 + 4 * k + 0.5f, qb, q2, bp.alpha_max, dx, dy, e)
                              : gauss_alpha(fx, py0 + 4 * k + 0.5f, qb, bp.alpha_max, dx, dy, d2, e);
        if (a < bp.alpha_min) continue;
        const float test = T[k] * (1.f - a);
        if (test < bp.t_min) {
          done[k] = true;
          stop[k] = base + b + 1;
          continue;
        }
        const float wgt = a * T[k];
        const float4 cc = s_c[w][b];
        acc[k][0] = fmaf(cc.x, wgt, acc[k][0]);
        if (C == 3) {
          acc[k][1] = fmaf(cc.y, wgt, acc[k][1]);
          acc[k][2] = fmaf(cc.z, wgt, acc[k][2]);
        }
        T[k] = test;
        last[k] = base + b + 1;
        ++contribs;
      }
      if (all_done()) m = 0;
    }
    __syncwarp();
  }
  count_evals(&st->blend_evals, evals);
  count_evals(&st->blend_contribs, contribs);
  unsigned int visits = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k)
    if (px < bp.W && py0 + 4 * k < bp.H) visits += stop[k] ? stop[k] : n;
  count_evals(&st->blend_visits, visits);
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int py = py0 + 4 * k;
    if (px < bp.W && py < bp.H) {
      const long long pix = ((long long)s * bp.H + py) * bp.W + px;
      float* out = image + pix * C;
      out[0] = acc[k][0] + T[k] * bp.bg0;
      if (C == 3) {
        out[1] = acc[k][1] + T[k] * bp.bg1;
        out[2] = acc[k][2] + T[k] * bp.bg2;
      }
      Tfinal[pix] = T[k];
      nlast[pix] = last[k];
    }
  }
}

template <int TILE, int PPT, int C, bool ANISO>
__global__ void __launch_bounds__(BlendGeom<TILE, PPT>::kThreads, BlendGeom<TILE, PPT>::kMinBlocksBwd)
    k_blend_bwd_groups(const int2* __restrict__ ranges, const uint32_t* __restrict__ gid,
                       const float4* __restrict__ prep, const float2* __restrict__ prep2,
                       const float2* __restrict__ reach, const int* __restrict__ gcurve,
                       const float4* __restrict__ color, BlendParams bp, const float* __restrict__ dimage,
                       const float* __restrict__ Tfinal, const int* __restrict__ nlast, float* dgauss, DevState* st,
                       int full_grads, float* /* per-curve colour gradients: unused, the rows carry them */) {
  grid_dep_wait();
  using Gm = BlendGeom<TILE, PPT>;
  constexpr int kRow = GradRow<ANISO>::kFloats;
  __shared__ float4 s_q[Gm::kWarps][32];
  __shared__ float4 s_c[Gm::kWarps][32];
  __shared__ float s_isig[Gm::kWarps][32];
  __shared__ uint32_t s_id[Gm::kWarps][32];
  __shared__ float2 s_q2[ANISO ? Gm::kWarps : 1][32];
  int s, px, py0;
  float bxf, y0, y1;
  group_pixels<TILE, PPT>(bp, s, px, py0, bxf, y0, y1);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, gi = lane & 7;
  const float fx = px + 0.5f;
  const int2 rg = ranges[blockIdx.x];
  float T[PPT], dI[PPT][3], Bk[PPT][3];
  int last[PPT];
  int gmax = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int py = py0 + 4 * k;
    T[k] = 1.f;
    last[k] = 0;
    Bk[k][0] = bp.bg0;
    Bk[k][1] = bp.bg1;
    Bk[k][2] = bp.bg2;
    dI[k][0] = dI[k][1] = dI[k][2] = 0.f;
    if (px < bp.W && py < bp.H) {
      const long long pix = ((long long)s * bp.H + py) * bp.W + px;
      T[k] = Tfinal[pix];
      last[k] = nlast[pix];
#pragma unroll
      for (int ch = 0; ch < C; ++ch) dI[k][ch] = dimage[pix * C + ch];
    }
    gmax = max(gmax, last[k]);
  }
  // list length of the group (its masks are trimmed to it, so that all eight
  // lanes pop the same entries) and of the warp
  for (int o = 4; o > 0; o >>= 1) gmax = max(gmax, __shfl_xor_sync(0xffffffffu, gmax, o));
  int wmax = gmax;
  for (int o = 16; o > 4; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  unsigned int evals = 0;
  for (int base = ((wmax - 1) >> 5) << 5; base >= 0 && wmax > 0; base -= 32) {
    const int j = base + lane;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 rs = make_float2(-1.f, 0.f);
    uint32_t g = 0;
    if (j < wmax) {
      g = gid[rg.x + j];
      if (!(g & kLayerBit)) {   // fill-layer entries (settings of another pass) are never read here
        q = prep[g];
        rs = reach[g];
      }
    }
    bool hit;
    unsigned int m = group_masks(j < wmax, q.x, q.y, rs.x, bxf, y0, y1, hit);
    if (hit) {
      s_q[w][lane] = q;
      s_c[w][lane] = color[gcurve[g]];
      s_isig[w][lane] = rs.y;
      s_id[w][lane] = g;
      if (ANISO) s_q2[ANISO ? w : 0][lane] = prep2[g];
    }
    const int lim = gmax - base;
    m &= lim >= 32 ? 0xffffffffu : (lim <= 0 ? 0u : ((1u << lim) - 1u));
    __syncwarp();
    while (__any_sync(0xffffffffu, m != 0)) {
      const bool act = m != 0;
      int b = 0;
      float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      float vC = 0.f;   // dC of a tangent-aligned Gaussian
      bool contrib = false, geo = false;
      if (act) {
        b = 31 - __clz(m);
        m &= ~(1u << b);
        const float4 qb = s_q[w][b];
        const float2 q2 = ANISO ? s_q2[ANISO ? w : 0][b] : make_float2(0.f, 0.f);
        const float isg_raw = s_isig[w][b];
        // fill Gaussians (negative 1/sigma) need only the opacity and colour
        // gradients unless the caller asked for every per-Gaussian gradient
        geo = full_grads || isg_raw > 0.f;
        const float isg = fabsf(isg_raw);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (base + b >= last[k]) continue;
          ++evals;
          float dx, dy, d2 = 0.f, e;
          const float a = ANISO ? gauss_alpha_aniso(fx, py0 + 4 * k + 0.5f, qb, q2, bp.alpha_max, dx, dy, e)
                                : gauss_alpha(fx, py0 + 4 * k + 0.5f, qb, bp.alpha_max, dx, dy, d2, e);
          if (a < bp.alpha_min) continue;
          contrib = true;
          T[k] = __fdividef(T[k], 1.f - a);   // transmittance in front of this Gaussian
          const float wgt = a * T[k];
          const float4 cc = s_c[w][b];
          float da = (cc.x - Bk[k][0]) * dI[k][0];
          v[5] += wgt * dI[k][0];
          Bk[k][0] = a * cc.x + (1.f - a) * Bk[k][0];
          if (C == 3) {
            da += (cc.y - Bk[k][1]) * dI[k][1] + (cc.z - Bk[k][2]) * dI[k][2];
            v[6] += wgt * dI[k][1];
            v[7] += wgt * dI[k][2];
            Bk[k][1] = a * cc.y + (1.f - a) * Bk[k][1];
            Bk[k][2] = a * cc.z + (1.f - a) * Bk[k][2];
          }
          da *= T[k];
          if (__fmul_rn(qb.w, e) < bp.alpha_max) {
            v[4] += e * da;
            if (geo) {
              if (ANISO) {
                const float ga = da * a;
                v[0] -= ga * (2.f * qb.z * dx + q2.x * dy);
                v[1] -= ga * (q2.x * dx + 2.f * q2.y * dy);
                v[2] += ga * dx * dx;
                v[3] += ga * dx * dy;
                vC += ga * dy * dy;
              } else {
                const float aa = da * a * isg * isg;
                v[0] += aa * dx;
                v[1] += aa * dy;
                v[2] += aa * d2 * isg;
              }
            }
          }
        }
      }
      // per-group reductions: every lane takes part in the shuffles, the
      // group's lanes 0 (and 4) write its Gaussian's row
      const unsigned int cb = __ballot_sync(0xffffffffu, contrib);
      const bool gcontrib = ((cb >> (lane & 24)) & 0xffu) != 0u;
      if (cb == 0u) continue;   // no group composited anything: nothing to reduce
      if (__any_sync(0xffffffffu, contrib && geo)) {
        const float t = group_sum8(v);
        const float t1 = __shfl_down_sync(0xffffffffu, t, 1, 8);
        const float t2 = __shfl_down_sync(0xffffffffu, t, 2, 8);
        const float t3 = __shfl_down_sync(0xffffffffu, t, 3, 8);
        if (ANISO) {
          float tc = vC;
          for (int o = 4; o > 0; o >>= 1) tc += __shfl_xor_sync(0xffffffffu, tc, o);
          if (gcontrib && geo && gi == 0 && tc != 0.f) atomicAdd(dgauss + (long long)s_id[w][b] * kRow + 8, tc);
        }
        if (gcontrib && (gi == 4 || (gi == 0 && geo)))
          red_add_v4(dgauss + (long long)s_id[w][b] * kRow + gi, t, t1, t2, t3);
      } else {
        const float t = group_sum4(v + 4);
        const float t1 = __shfl_down_sync(0xffffffffu, t, 2, 8);
        const float t2 = __shfl_down_sync(0xffffffffu, t, 4, 8);
        const float t3 = __shfl_down_sync(0xffffffffu, t, 6, 8);
        if (gcontrib && gi == 0) red_add_v4(dgauss + (long long)s_id[w][b] * kRow + 4, t, t1, t2, t3);
      }
    }
    __syncwarp();
  }
  count_evals(&st->blend_bwd_evals, evals);
  unsigned int visits = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) visits += last[k];
  count_evals(&st->blend_bwd_visits, visits);
}

// (TILE, decomposition) -> launch.  Valid: TILE 8 with PPT 1-2, TILE 16 and 32 with PPT 1-4; lane groups
// with PPT 1-2 at every tile.
// ---------------------------------------------------------------------------
// Fill layers (ns_raster_params.fill_layers, isotropic sets).  The Gaussians
// of a filled curve sit on its grid (§3.3): record g_off + iy nx + ix is grid
// point (ix, iy), and all share one sigma.  The binning then emits one pair
// per tile of the whole layer (value g_off | kLayerBit).  On such an entry a
// pixel composites, in sample order, the grid points that can reach it:
//   - the columns and rows whose bin rectangle covers this tile, by the exact
//     float32 rule of tile_rect (the Gaussians per-Gaussian pairs would list);
//     k_layer_runs finds these runs once per forward, per curve and tile
//     column or row;
//   - narrowed, when alpha_min > 0, to |q - p| <= R per axis, R the reach of
//     the layer's most opaque Gaussian (beyond it alpha < alpha_min);
//   - skipping the grid points tile_rect would not bin (culled opacity).
// A pixel thus composites exactly the Gaussians, in the order and with the
// arithmetic of the per-Gaussian lists, and the image is the same bit for
// bit.  Each warp stages the records of the grid points its pixels can see
// (its region) in shared memory with coalesced loads, culled points marked,
// and skips a layer whose region holds no live point.  The adjoint also
// needs, per pixel, the sample index of the last composited Gaussian inside
// its layer (nsub) besides the list position.

struct LayerArgs {
  const CurvePlan* plan;
  const float4* rec;
  const int* gcount;
  const int2* runs;   // per curve: covered column run per tile column, then row run per tile row
  const float4* lconst;   // per curve: {X0, Y0, xoff, yoff}, {sigma, ncoef log2(e), nx bits, ny bits},
                          // {h, 1/h, R, 0}
                          // with the grid origin X0 + xoff (X0 an integer), from k_layer_runs
  int gcap, tile, tiles_x, runs_stride;
  float k_sigma, inv_tile, log_amin;
  int* nsub;   // per pixel: 1 + sample index of the last composited fill Gaussian (0: none)
  float* dop;  // the adjoint's opacity gradients of layer points, one float per Gaussian (NULL: entry 4
               // of the Gaussian's gradient row)
};

// Where the adjoint adds the opacity gradient of grid point g of a fill layer.
__device__ __forceinline__ float* layer_dop(const LayerArgs& la, float* dgauss, long long g, int row) {
  return la.dop ? la.dop + g : dgauss + g * row + 4;
}

// One layer as a warp sees it on one tile (the same in every lane).
struct LayerView {
  long long g_off, G;   // first Gaussian; Gaussians in the set (nothing at or past G is read)
  int nx, ny;
  float x0, y0, inv_h, sig, nc2, R;   // x0, y0: the grid origin rounded to float (windows only);
                                      // nc2 = -log2(e) / (2 sigma^2)
  float X0, Y0, xoff, yoff, h;       // the origin as integer + offset, for the exact local offsets
  int cx0, cx1, cy0, cy1;   // columns and rows binned to this tile (empty when cx0 > cx1)
};

__device__ __forceinline__ bool bin_covers(float v, float ks, float inv_tile, int t) {
  return floorf(__fmul_rn(__fsub_rn(v, ks), inv_tile)) <= float(t) &&
         float(t) <= floorf(__fmul_rn(__fadd_rn(v, ks), inv_tile));
}

// The run of indices in [0, n) where ok() holds (contiguous: a bin
// rectangle moves with its centre), found from a guess inside or near it.
template <typename F>
__device__ __forceinline__ void covered_run(int n, float guess, F ok, int& lo, int& hi) {
  lo = 0;
  hi = -1;
  if (n <= 0) return;
  int i = int(fminf(fmaxf(guess, 0.f), float(n - 1)));
  if (!ok(i)) {
    int a = i - 1, b = i + 1;
    bool found = false;
    while (!found && (a >= 0 || b < n)) {
      if (b < n && ok(b)) {
        i = b;
        found = true;
      } else if (a >= 0 && ok(a)) {
        i = a;
        found = true;
      }
      --a;
      ++b;
    }
    if (!found) return;
  }
  lo = hi = i;
  while (lo > 0 && ok(lo - 1)) --lo;
  while (hi + 1 < n && ok(hi + 1)) ++hi;
}

// The same run from arithmetic guesses of both ends (g_lo, g_hi: the real
// bounds of the indices whose grid coordinate the bin rule puts on the tile),
// confirmed by four independent reads: the ends hold and their outer
// neighbours do not.  The walk above when the check fails.
template <typename F>
__device__ __forceinline__ void covered_run_guess(int n, float g_lo, float g_hi, F ok, int& lo, int& hi) {
  if (n > 0) {
    const int a = max(int(ceilf(fminf(fmaxf(g_lo, -1.f), float(n)))), 0);
    const int b = min(int(ceilf(fminf(fmaxf(g_hi, -1.f), float(n + 1)))) - 1, n - 1);
    if (a <= b) {
      const bool in_a = ok(a), in_b = ok(b), in_am = ok(max(a - 1, 0)), in_bp = ok(min(b + 1, n - 1));
      if (in_a && in_b && (a == 0 || !in_am) && (b == n - 1 || !in_bp)) {
        lo = a;
        hi = b;
        return;
      }
    }
  }
  covered_run(n, g_lo, ok, lo, hi);
}

// One block per curve: for each tile column (row) of a fill layer's tile
// rectangle, the run of grid columns (rows) the bin rule puts on it.
// Thread 0 also writes the layer's constants: origin, 1/h, the reach bound R
// of its most opaque Gaussian (+inf when alpha_min = 0), sigma and the
// exponent coefficient the per-Gaussian binning would prepare.
__global__ void __launch_bounds__(128) k_layer_runs(ns_curves cv, const CurvePlan* __restrict__ plan,
                                                    const float4* __restrict__ rec, const int* __restrict__ gcount,
                                                    BinParams bp, int2* runs, int stride, float4* lconst,
                                                    const float2* __restrict__ glo) {
  grid_dep_wait();
  const int c = blockIdx.x;
  if (!(cv.flags[c] & NS_FILLED)) return;
  const CurvePlan p = plan[c];
  const long long G = min((long long)*gcount, (long long)bp.gcap);
  if (p.g_off < 0 || p.g_off >= G || p.count <= 0 || p.nx <= 0 || p.ny <= 0 || !(p.h > 0.f)) return;
  if (threadIdx.x == 0) {
    const float sig = rec[p.g_off].z;
    const float o_c = cv.color[4 * c + 3];
    const float R = !(o_c > 0.f) ? 0.f
                    : (bp.log_amin > -1e30f ? sqrtf(reach2(sig, o_c, bp.log_amin)) + 0.01f * p.h : FLT_MAX);
    // origin = X0 + xoff with X0 an integer: pixel centre - X0 is exact, and
    // xoff (the fraction plus the low part of nurbs_sample's FP64 origin) keeps
    // the offset of a pixel from a grid point exact to ~1e-7 px at any canvas size
    const float2 lo = glo[c];
    const float X0 = floorf(p.x0), Y0 = floorf(p.y0);
    lconst[3 * c] = make_float4(X0, Y0, __fadd_rn(__fsub_rn(p.x0, X0), lo.x), __fadd_rn(__fsub_rn(p.y0, Y0), lo.y));
    lconst[3 * c + 1] = make_float4(sig, ncoef2(sig), __int_as_float(p.nx), __int_as_float(p.ny));
    lconst[3 * c + 2] = make_float4(p.h, 1.f / p.h, R, 0.f);
  }
  int tx0, ty0, ntx;
  const int nt = layer_rect_live(rec, p, G, bp, c, tx0, ty0, ntx);
  if (!nt) return;
  const int2 live0 = bp.lmin[c], live1 = bp.lmax[c];   // runs keep to the live columns and rows
  const int nty = nt / ntx;
  const float ks = __fmul_rn(bp.k_sigma, rec[p.g_off].z);
  const float inv_h = 1.f / p.h, T = 1.f / bp.inv_tile;
  const long long lastg = G - 1;
  int2* out = runs + (long long)c * stride;
  for (int k = threadIdx.x; k < ntx + nty; k += blockDim.x) {
    int lo, hi;
    if (k < ntx) {
      const int tx = tx0 + k;
      covered_run_guess(p.nx, (tx * T - ks - p.x0) * inv_h - 0.5f, ((tx + 1) * T + ks - p.x0) * inv_h - 0.5f,
                        [&](int ix) { return bin_covers(rec[min((long long)p.g_off + ix, lastg)].x, ks, bp.inv_tile, tx); },
                        lo, hi);
      out[tx] = make_int2(max(lo, live0.x), min(hi, live1.x));
    } else {
      const int ty = ty0 + (k - ntx);
      covered_run_guess(p.ny, (ty * T - ks - p.y0) * inv_h - 0.5f, ((ty + 1) * T + ks - p.y0) * inv_h - 0.5f,
                        [&](int iy) {
                          return bin_covers(rec[min((long long)p.g_off + (long long)iy * p.nx, lastg)].y, ks,
                                            bp.inv_tile, ty);
                        },
                        lo, hi);
      out[bp.tiles_x + ty] = make_int2(max(lo, live0.y), min(hi, live1.y));
    }
  }
}

// The layer of curve c (first Gaussian g_off) on tile (tx, ty); empty when
// the curve's constants were not written (nothing to composite).
// What a layer entry needs from global memory, loaded by the lane that loads
// the entry of a list batch: the layer constants and the grid runs of the
// tile ({column run, row run}).
__device__ __forceinline__ void layer_entry(const LayerArgs& la, int c, int tx, int ty, float4& k0, float4& k1,
                                            float4& k2, int4& run) {
  k0 = la.lconst[3 * c];
  k1 = la.lconst[3 * c + 1];
  k2 = la.lconst[3 * c + 2];
  const int2* r = la.runs + (long long)c * la.runs_stride;
  const int2 rx = r[tx], ry = r[la.tiles_x + ty];
  run = make_int4(rx.x, rx.y, ry.x, ry.y);
}

__device__ __forceinline__ LayerView layer_view(const float4& k0, const float4& k1, const float4& k2,
                                                const int4& run, long long g_off, long long G) {
  LayerView v;
  const int2 rx = make_int2(run.x, run.y), ry = make_int2(run.z, run.w);
  v.G = G;
  v.g_off = g_off;
  v.X0 = k0.x;
  v.Y0 = k0.y;
  v.xoff = k0.z;
  v.yoff = k0.w;
  v.x0 = k0.x + k0.z;
  v.y0 = k0.y + k0.w;
  v.h = k2.x;
  v.inv_h = k2.y;
  v.R = k2.z;
  v.sig = k1.x;
  v.nc2 = k1.y;
  v.nx = __float_as_int(k1.z);
  v.ny = __float_as_int(k1.w);
  v.cx0 = rx.x;
  v.cx1 = rx.y;
  v.cy0 = ry.x;
  v.cy1 = ry.y;
  if (!(v.R > 0.f) || v.nx <= 0 || v.ny <= 0) {
    v.cx0 = v.cy0 = 0;
    v.cx1 = v.cy1 = -1;
  }
  return v;
}

// The grid points of the layer one pixel (centre fx, fy) may see.
__device__ __forceinline__ void layer_window(const LayerView& v, float fx, float fy, int& ix0, int& ix1, int& iy0,
                                             int& iy1) {
  ix0 = v.cx0;
  ix1 = v.cx1;
  iy0 = v.cy0;
  iy1 = v.cy1;
  if (v.R < FLT_MAX) {
    ix0 = max(ix0, int(ceilf(fmaxf((fx - v.R - v.x0) * v.inv_h - 0.5f, -1.f))));
    ix1 = min(ix1, int(floorf(fminf((fx + v.R - v.x0) * v.inv_h - 0.5f, 2e9f))));
    iy0 = max(iy0, int(ceilf(fmaxf((fy - v.R - v.y0) * v.inv_h - 0.5f, -1.f))));
    iy1 = min(iy1, int(floorf(fminf((fy + v.R - v.y0) * v.inv_h - 0.5f, 2e9f))));
  }
}

// Grid-local coordinate of grid column (row) i, as nurbs_sample placed it.
__device__ __forceinline__ float layer_qx(const LayerView& v, int i) { return (float(i) + 0.5f) * v.h; }

// The offset of grid row iy from the pixel row whose centre minus the integer
// origin is fyl: (fyl - qy) - yoff, exact to ~1e-7 px.  It is the same for
// every point of the row, so the walks form it (and its square) once per row.
__device__ __forceinline__ float layer_dy(const LayerView& v, float fyl, int iy) {
  return __fsub_rn(__fsub_rn(fyl, layer_qx(v, iy)), v.yoff);
}

// The warp's region of a layer: the grid points the pixel centres of its
// rectangle wr = (x0, x1, y0, y1) can see.  It contains every pixel's
// window (the bounds are monotone in the pixel position); false if empty.
__device__ __forceinline__ bool layer_region(const LayerView& v, const float4& wr, int& rx0, int& rx1, int& ry0,
                                             int& ry1) {
  rx0 = v.cx0;
  rx1 = v.cx1;
  ry0 = v.cy0;
  ry1 = v.cy1;
  if (v.R < FLT_MAX) {
    rx0 = max(rx0, int(ceilf(fmaxf((wr.x - v.R - v.x0) * v.inv_h - 0.5f, -1.f))));
    rx1 = min(rx1, int(floorf(fminf((wr.y + v.R - v.x0) * v.inv_h - 0.5f, 2e9f))));
    ry0 = max(ry0, int(ceilf(fmaxf((wr.z - v.R - v.y0) * v.inv_h - 0.5f, -1.f))));
    ry1 = min(ry1, int(floorf(fminf((wr.w + v.R - v.y0) * v.inv_h - 0.5f, 2e9f))));
  }
  return rx1 >= rx0 && ry1 >= ry0;
}

// What a warp keeps per fill-layer entry of a list batch, prepared by the
// lane that loads the entry (the 32 entries of a batch in parallel): the
// region of grid points the warp's pixel rectangle wr can see (rx0 > rx1:
// none), and the layer's constants for the pixels' windows and the walk.
// Fill Gaussians of one curve share sigma (eta h / rho, Eq. 6), so a layer
// has one exponent coefficient.
__device__ __forceinline__ void layer_prepare(const LayerArgs& la, int c, int tx, int ty, const float4& wr,
                                              int4& reg, float4& win, float4& loc, float4& org) {
  float4 k0, k1, k2;
  int4 run;
  layer_entry(la, c, tx, ty, k0, k1, k2, run);
  const LayerView v = layer_view(k0, k1, k2, run, 0, 0);
  int rx0, rx1, ry0, ry1;
  if (!(v.sig > 0.f) || !layer_region(v, wr, rx0, rx1, ry0, ry1)) {
    rx0 = ry0 = 1;
    rx1 = ry1 = 0;
  }
  reg = make_int4(rx0, rx1, ry0, ry1);
  win = make_float4(v.x0, v.y0, v.inv_h, v.R);
  loc = make_float4(v.xoff, v.yoff, v.h, v.nc2);
  org = make_float4(v.X0, v.Y0, __int_as_float(v.nx), v.sig);
}

// The layer as the warp sees it, from the prepared entry: the region's bounds
// stand in for the tile's runs (every pixel window lies inside the region,
// and both clamp to the runs and the reach the same way).
__device__ __forceinline__ LayerView layer_unpack(const int4& reg, const float4& win, const float4& loc,
                                                  const float4& org, long long g_off, long long G) {
  LayerView v;
  v.g_off = g_off;
  v.G = G;
  v.x0 = win.x;
  v.y0 = win.y;
  v.inv_h = win.z;
  v.R = win.w;
  v.xoff = loc.x;
  v.yoff = loc.y;
  v.h = loc.z;
  v.nc2 = loc.w;
  v.X0 = org.x;
  v.Y0 = org.y;
  v.nx = __float_as_int(org.z);
  v.sig = org.w;
  v.ny = 0;
  v.cx0 = reg.x;
  v.cx1 = reg.y;
  v.cy0 = reg.z;
  v.cy1 = reg.w;
  return v;
}

// alpha of a staged grid point {qx, o} (o < 0: not listed) at the pixel whose
// centre minus the integer origin has x part fxl, on a row at squared offset
// dy2 (as layer_alpha, with the layer's coefficient).
__device__ __forceinline__ float layer_alpha_o(const LayerView& v, float fxl, float dy2, const float2& q, float amax,
                                               float& dx, float& d2, float& e) {
  dx = __fsub_rn(__fsub_rn(fxl, q.x), v.xoff);
  d2 = __fmaf_rn(dx, dx, dy2);
  e = ex2_approx(__fmul_rn(v.nc2, d2));
  return fminf(__fmul_rn(q.y, e), amax);
}

// A grid point of opacity o the per-Gaussian binning would list (sigma > 0
// is checked once per layer).
__device__ __forceinline__ bool layer_o_binned(float o, float alpha_min) { return o > 0.f && o >= alpha_min; }

// Asynchronous 4-byte copy from global to shared memory (cp.async; bytes past
// src_bytes are zero-filled), its group commit and the wait for all groups.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int src_bytes) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Requests a layer region (reg, of at most 32 kIt points) as {qx, o}: the
// grid coordinates are written at once, the opacities arrive by cp.async
// (0 past the Gaussian set).  The caller commits the group and waits for it
// before reading.
template <int kIt>
__device__ __forceinline__ void layer_prefetch(const LayerArgs& la, long long g_off, long long G, int nx, float h,
                                               const int4& reg, float2* pts) {
  const int lane = threadIdx.x & 31;
  const int rw = reg.y - reg.x + 1, npt = rw * (reg.w - reg.z + 1);
  const float inv_rw = __fdividef(1.f, float(rw));   // the quotients below stay 0.5/rw off integers
  const float* op = reinterpret_cast<const float*>(la.rec) + 3;   // the records' opacities
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int i = lane + 32 * it;
    if (i < npt) {
      const int iyr = int((float(i) + 0.5f) * inv_rw);   // exact for the region sizes staged here
      const int ix = reg.x + (i - iyr * rw);
      const long long g = g_off + (long long)(reg.z + iyr) * nx + ix;
      pts[i].x = (float(ix) + 0.5f) * h;
      const bool in = g < G;
      cp_async4(&pts[i].y, op + 4 * (in ? g : 0), in ? 4 : 0);
    }
  }
}

// Requests entry b of a warp's batch (a staged fill layer) into pts.
template <int kIt>
__device__ __forceinline__ void layer_request(const LayerArgs& la, long long G, const uint32_t* ids, const int4* regs,
                                              const float4* locs, const float4* orgs, int b, float2* pts) {
  layer_prefetch<kIt>(la, ids[b] & ~kLayerBit, G, __float_as_int(orgs[b].z), locs[b].z, regs[b], pts);
  cp_async_commit();
}

// Whether any point of a staged region is one the per-Gaussian binning would
// list (the same in every lane).
template <int kIt>
__device__ __forceinline__ bool layer_live(const float2* pts, int npt, float alpha_min) {
  const int lane = threadIdx.x & 31;
  bool live = false;
#pragma unroll
  for (int it = 0; it < kIt; ++it) {
    const int i = lane + 32 * it;
    if (i < npt) live = live || layer_o_binned(pts[i].y, alpha_min);
  }
  return __any_sync(0xffffffffu, live);
}

// The next entry of a batch (bits of mask, lowest first, or highest first for
// the adjoint) that is a fill layer with a region of at most kPts points, or -1.
template <int kPts, bool kHighFirst>
__device__ __forceinline__ int next_staged_layer(unsigned int mask, const uint32_t* ids, const int4* regs) {
  while (mask) {
    const int b = kHighFirst ? 31 - __clz(mask) : __ffs(mask) - 1;
    mask &= ~(1u << b);
    if (ids[b] & kLayerBit) {
      const int4 r = regs[b];
      if ((long long)(r.y - r.x + 1) * (r.w - r.z + 1) <= kPts) return b;
    }
  }
  return -1;
}

template <int TILE, int PPT>
struct LayerGeom {
  // staged points per warp; the forward and the adjoint share a budget of
  // shared memory per block that keeps every instantiation under 48 KB
  static constexpr int kPts = BlendGeom<TILE, PPT>::kWarps <= 2 ? 192 : 128;
  // 1024 resident threads (64 registers): the adjoint is latency-bound, and
  // 16 blocks of 2 warps per SM beat 12 blocks at 80 registers (a few bytes
  // of spills outside the walk)
  static constexpr int kMinBlocksBwd = 1024 / BlendGeom<TILE, PPT>::kThreads;
  // the forward at 56 registers: 18 blocks of 2 warps per SM; blocks of one
  // warp (two pixels per thread) at 80 registers, 24 blocks per SM (at 64
  // registers, 32 blocks, their pixel state spills)
  static constexpr int kMinBlocksFwd =
      1152 / BlendGeom<TILE, PPT>::kThreads < 32 ? 1152 / BlendGeom<TILE, PPT>::kThreads : 24;
};

template <int TILE, int PPT, int C>
__global__ void __launch_bounds__(BlendGeom<TILE, PPT>::kThreads, LayerGeom<TILE, PPT>::kMinBlocksFwd)
    k_blend_fwd_layers(const int2* __restrict__ ranges, const uint32_t* __restrict__ gid,
                       const float4* __restrict__ prep, const float2* __restrict__ reach,
                       const int* __restrict__ gcurve, const float4* __restrict__ color, BlendParams bp,
                       LayerArgs la, float* image, float* Tfinal, int* nlast, DevState* st) {
  grid_dep_wait();
  using Gm = BlendGeom<TILE, PPT>;
  constexpr int kPts = LayerGeom<TILE, PPT>::kPts;
  __shared__ float4 s_q[Gm::kWarps][32];     // blend constants, or a layer's {xoff, yoff, h, nc2}
  __shared__ float4 s_c[Gm::kWarps][32];
  __shared__ uint32_t s_id[Gm::kWarps][32];
  __shared__ float4 s_win[Gm::kWarps][32];   // a layer's {x0, y0, 1/h, R}
  __shared__ float4 s_org[Gm::kWarps][32];   // a layer's {X0, Y0, nx bits, sigma}
  __shared__ int4 s_rg[Gm::kWarps][32];      // a layer's region for this warp
  __shared__ float2 s_pt[Gm::kWarps][2][kPts];   // staged regions: the current entry's and the next one's
  int s, px, py0;
  float4 wr;
  tile_pixels<TILE, PPT>(bp, s, px, py0, wr);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x - s * bp.tiles_per_scene;
  const int tx = t % bp.tiles_x, ty = t / bp.tiles_x;
  const float fx = px + 0.5f;
  const int2 rg = ranges[blockIdx.x];
  const long long Gset = min((long long)*la.gcount, (long long)la.gcap);   // Gaussians in the set
  const int n = rg.y - rg.x;
  float T[PPT], acc[PPT][C];
  bool done[PPT];
  int last[PPT], lsub[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    T[k] = 1.f;
    done[k] = !(px < bp.W && py0 + 4 * k < bp.H);
    last[k] = 0;
    lsub[k] = 0;
#pragma unroll
    for (int ch = 0; ch < C; ++ch) acc[k][ch] = 0.f;
  }
  auto all_done = [&]() {
    bool d = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) d = d && done[k];
    return d;
  };
  unsigned int evals = 0, contribs = 0;
  int cur = 0;   // the buffer holding the current staged entry's region
  // composite one Gaussian (blend constants q) into pixel k; false once the pixel is done
  // the compositing step of Eq. 8 once alpha is known
  auto composite_alpha = [&](int k, float a, const float4& cc, int pos, int sub) {
    ++evals;
    if (a < bp.alpha_min) return;
    const float test = T[k] * (1.f - a);
    if (test < bp.t_min) {
      done[k] = true;
      return;
    }
    const float wgt = a * T[k];
    acc[k][0] = fmaf(cc.x, wgt, acc[k][0]);
    if (C == 3) {
      acc[k][1] = fmaf(cc.y, wgt, acc[k][1]);
      acc[k][2] = fmaf(cc.z, wgt, acc[k][2]);
    }
    T[k] = test;
    last[k] = pos;
    lsub[k] = sub;
    ++contribs;
  };
  auto composite = [&](int k, float fy, const float4& q, const float4& cc, int pos, int sub) {
    float dx, dy, d2, e;
    composite_alpha(k, gauss_alpha(fx, fy, q, bp.alpha_max, dx, dy, d2, e), cc, pos, sub);
  };
  // the same step for grid point (column ix) of a layer: every point of the
  // layer has the curve's colour, so the weights a T of Eq. 8 are summed
  // (wsum) and the colour is added once per layer; the walk counts its
  // evaluations per row and records the row's last composited column (lix)
  auto composite_layer = [&](int k, float a, float& wsum, int ix, int& lix) {
    if (a < bp.alpha_min) return;
    const float test = T[k] * (1.f - a);
    if (test < bp.t_min) {
      done[k] = true;
      return;
    }
    wsum = fmaf(a, T[k], wsum);
    T[k] = test;
    lix = ix;
    ++contribs;
  };
  // the same without branches for a staged point of opacity o (o <= 0: not
  // listed), after which pixel k may be done
  auto composite_point = [&](int k, float a, float o, float& wsum, int ix, int& lix) {
    const bool ok = o > 0.f && a >= bp.alpha_min && !done[k];
    const float test = T[k] * (1.f - a);
    const bool stop = ok && test < bp.t_min;
    const bool comp = ok && !stop;
    done[k] = done[k] || stop;
    wsum = comp ? fmaf(a, T[k], wsum) : wsum;
    T[k] = comp ? test : T[k];
    lix = comp ? ix : lix;
    contribs += comp ? 1u : 0u;
  };
  for (int base = 0; base < n && !__all_sync(0xffffffffu, all_done()); base += 32) {
    const int j = base + lane;
    bool hit = false;
    if (j < n) {
      const uint32_t g = gid[rg.x + j];
      const uint32_t gi = g & ~kLayerBit;
      if (g & kLayerBit) {
        const int c = gcurve[gi];
        int4 reg;
        float4 win, loc, org;
        layer_prepare(la, c, tx, ty, wr, reg, win, loc, org);
        hit = reg.x <= reg.y;
        if (hit) {
          s_id[w][lane] = g;
          s_c[w][lane] = color[c];
          s_q[w][lane] = loc;
          s_win[w][lane] = win;
          s_org[w][lane] = org;
          s_rg[w][lane] = reg;
        }
      } else {
        const float4 q = prep[gi];
        hit = rect_d2(q.x, q.y, wr.x, wr.y, wr.z, wr.w) <= reach[gi].x;
        if (hit) {
          s_id[w][lane] = g;
          s_q[w][lane] = q;
          s_c[w][lane] = color[gcurve[gi]];
        }
      }
    }
    unsigned int mask = __ballot_sync(0xffffffffu, hit);
    __syncwarp();
    // the first staged layer entry's region is requested now; each staged
    // entry requests the next one's before its own walk
    {
      const int nb = next_staged_layer<kPts, false>(mask, s_id[w], s_rg[w]);
      if (nb >= 0) layer_request<kPts / 32>(la, Gset, s_id[w], s_rg[w], s_q[w], s_org[w], nb, s_pt[w][cur]);
    }
    while (mask) {
      const int b = __ffs(mask) - 1;
      mask &= mask - 1;
      const uint32_t id = s_id[w][b];
      const float4 cc = s_c[w][b];
      if (id & kLayerBit) {
        if (!__any_sync(0xffffffffu, !all_done())) break;
        const uint32_t g0 = id & ~kLayerBit;
        const int4 reg = s_rg[w][b];
        const LayerView v = layer_unpack(reg, s_win[w][b], s_q[w][b], s_org[w][b], g0, Gset);
        const float fxl = __fsub_rn(fx, v.X0);
        const int rx0 = reg.x, ry0 = reg.z;
        const int rw = reg.y - reg.x + 1, rh = reg.w - reg.z + 1;
        const bool staged = (long long)rw * rh <= kPts;
        if (staged) {
          cp_async_wait_all();
          __syncwarp();
          const int nb = next_staged_layer<kPts, false>(mask, s_id[w], s_rg[w]);
          if (nb >= 0) layer_request<kPts / 32>(la, Gset, s_id[w], s_rg[w], s_q[w], s_org[w], nb, s_pt[w][cur ^ 1]);
          if (!layer_live<kPts / 32>(s_pt[w][cur], rw * rh, bp.alpha_min)) {
            cur ^= 1;
            continue;
          }
        }
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (done[k]) continue;
          const float fy = py0 + 4 * k + 0.5f;
          const float fyl = __fsub_rn(fy, v.Y0);
          int ix0, ix1, iy0, iy1;
          layer_window(v, fx, fy, ix0, ix1, iy0, iy1);
          const int pos = base + b + 1;
          float wsum = 0.f;
          for (int iy = iy0; iy <= iy1 && !done[k]; ++iy) {
            const int rowsub = iy * v.nx;
            const float dy = layer_dy(v, fyl, iy), dy2 = __fmul_rn(dy, dy);
            int lix = -1;   // the row's last composited column
            if (staged) {
              // two points per step: both alphas are independent of the
              // compositing state, which then takes them in order
              const float2* prow = &s_pt[w][cur][(iy - ry0) * rw - rx0];
              int ix = ix0;
              for (; ix + 1 <= ix1 && !done[k]; ix += 2) {
                const float2 qa = prow[ix], qb = prow[ix + 1];
                float dx, d2, ea, eb;
                const float aa = layer_alpha_o(v, fxl, dy2, qa, bp.alpha_max, dx, d2, ea);
                const float ab = layer_alpha_o(v, fxl, dy2, qb, bp.alpha_max, dx, d2, eb);
                composite_point(k, aa, qa.y, wsum, ix, lix);
                composite_point(k, ab, qb.y, wsum, ix + 1, lix);
              }
              evals += ix - ix0;   // points whose alpha the loop formed
              if (ix <= ix1 && !done[k]) {
                const float2 q = prow[ix];
                float dx, d2, e;
                ++evals;
                composite_point(k, layer_alpha_o(v, fxl, dy2, q, bp.alpha_max, dx, d2, e), q.y, wsum, ix, lix);
              }
            } else {
              for (int ix = ix0; ix <= ix1 && !done[k]; ++ix) {
                const long long g = v.g_off + rowsub + ix;
                if (g >= v.G) break;
                const float o = la.rec[g].w;
                if (!layer_o_binned(o, bp.alpha_min)) continue;
                float dx, d2, e;
                ++evals;
                composite_layer(k, layer_alpha_o(v, fxl, dy2, make_float2(layer_qx(v, ix), o), bp.alpha_max, dx, d2, e),
                                wsum, ix, lix);
              }
            }
            if (lix >= 0) {
              last[k] = pos;
              lsub[k] = rowsub + lix + 1;
            }
          }
          acc[k][0] = fmaf(cc.x, wsum, acc[k][0]);
          if (C == 3) {
            acc[k][1] = fmaf(cc.y, wsum, acc[k][1]);
            acc[k][2] = fmaf(cc.z, wsum, acc[k][2]);
          }
        }
        if (staged) {
          __syncwarp();
          cur ^= 1;
        }
      } else {
        const float4 q = s_q[w][b];
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (done[k]) continue;
          composite(k, py0 + 4 * k + 0.5f, q, cc, base + b + 1, 0);
        }
      }
    }
    cp_async_wait_all();   // a request left behind by a warp whose pixels are done
    __syncwarp();
  }
  count_evals(&st->blend_evals, evals);
  count_evals(&st->blend_contribs, contribs);
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int py = py0 + 4 * k;
    if (px < bp.W && py < bp.H) {
      const long long pix = ((long long)s * bp.H + py) * bp.W + px;
      float* out = image + pix * C;
      out[0] = acc[k][0] + T[k] * bp.bg0;
      if (C == 3) {
        out[1] = acc[k][1] + T[k] * bp.bg1;
        out[2] = acc[k][2] + T[k] * bp.bg2;
      }
      Tfinal[pix] = T[k];
      nlast[pix] = last[k];
      la.nsub[pix] = lsub[k];
    }
  }
}

// The adjoint with fill layers.  Per layer entry the warp stages its region
// as the forward does; the opacity gradients of its grid points gather in a
// per-warp array of shared memory (shared atomics: at grid steps above 1 px
// neighbouring pixels see the same grid points) and go to the per-Gaussian
// rows once per layer, and the colour gradients of the layer are summed over
// the warp and added to the curve's.  When every per-Gaussian gradient is
// asked for, no per-curve output is given, or the region is too large to
// stage, each composited pair reads its record and adds its row directly.
template <int TILE, int PPT, int C>
__global__ void __launch_bounds__(BlendGeom<TILE, PPT>::kThreads, LayerGeom<TILE, PPT>::kMinBlocksBwd)
    k_blend_bwd_layers(const int2* __restrict__ ranges, const uint32_t* __restrict__ gid,
                       const float4* __restrict__ prep, const float2* __restrict__ reach,
                       const int* __restrict__ gcurve, const float4* __restrict__ color, BlendParams bp,
                       LayerArgs la, const float* __restrict__ dimage, const float* __restrict__ Tfinal,
                       const int* __restrict__ nlast, float* dgauss, DevState* st, int full_grads, float* dcurve) {
  grid_dep_wait();
  using Gm = BlendGeom<TILE, PPT>;
  constexpr int kRow = 8;
  constexpr int kPts = LayerGeom<TILE, PPT>::kPts;
  __shared__ float4 s_q[Gm::kWarps][32];     // blend constants, or a layer's {xoff, yoff, h, nc2}
  __shared__ float4 s_c[Gm::kWarps][32];
  __shared__ float s_isig[Gm::kWarps][32];   // +-1/sigma, or a layer's curve (int bits)
  __shared__ uint32_t s_id[Gm::kWarps][32];
  __shared__ float4 s_win[Gm::kWarps][32];   // a layer's {x0, y0, 1/h, R}
  __shared__ float4 s_org[Gm::kWarps][32];   // a layer's {X0, Y0, nx bits, sigma}
  __shared__ int4 s_rg[Gm::kWarps][32];      // a layer's region for this warp
  __shared__ float2 s_pt[Gm::kWarps][2][kPts];   // staged regions: the current entry's and the next one's
  // the opacity gradients of the current entry's region; zero between
  // entries (each flush clears what it reads)
  __shared__ __align__(16) float s_reg[Gm::kWarps][kPts];
  int s, px, py0;
  float4 wr;
  tile_pixels<TILE, PPT>(bp, s, px, py0, wr);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x - s * bp.tiles_per_scene;
  const int tx = t % bp.tiles_x, ty = t / bp.tiles_x;
  const float fx = px + 0.5f;
  const int2 rg = ranges[blockIdx.x];
  const long long Gset = min((long long)*la.gcount, (long long)la.gcap);   // Gaussians in the set
  const bool per_pair = full_grads || dcurve == nullptr;
  // S[k] = B . dI: the colour B composited behind the current pair (the
  // background first), projected on the pixel's image gradient; the opacity
  // adjoint needs only this projection (dL/dalpha = (c - B) . dI T)
  float T[PPT], dI[PPT][3], S[PPT];
  int last[PPT], lsub[PPT];
  int wmax = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int py = py0 + 4 * k;
    T[k] = 1.f;
    last[k] = 0;
    lsub[k] = 0;
    dI[k][0] = dI[k][1] = dI[k][2] = 0.f;
    if (px < bp.W && py < bp.H) {
      const long long pix = ((long long)s * bp.H + py) * bp.W + px;
      T[k] = Tfinal[pix];
      last[k] = nlast[pix];
      lsub[k] = la.nsub[pix];
#pragma unroll
      for (int ch = 0; ch < C; ++ch) dI[k][ch] = dimage[pix * C + ch];
    }
    S[k] = bp.bg0 * dI[k][0];
    if (C == 3) S[k] = fmaf(bp.bg2, dI[k][2], fmaf(bp.bg1, dI[k][1], S[k]));
    wmax = max(wmax, last[k]);
  }
  for (int o = 16; o > 0; o >>= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  for (int i = lane; i < kPts; i += 32) s_reg[w][i] = 0.f;
  __syncwarp();
  unsigned int evals = 0;
  // the adjoint of one pair of pixel k (blend constants q, colour cc):
  // returns false below alpha_min; else the opacity gradient dO, the colour
  // gradient col and, for the centre and sigma, da a and the offsets
  auto color_dot = [&](int k, const float4& cc) {
    float v = cc.x * dI[k][0];
    if (C == 3) v = fmaf(cc.z, dI[k][2], fmaf(cc.y, dI[k][1], v));
    return v;
  };
  auto adjoint_alpha = [&](int k, float a, float e, float ow, const float4& cc, float& dO, float col[3],
                           float& daa) {
    ++evals;
    if (a < bp.alpha_min) return false;
    T[k] = __fdividef(T[k], 1.f - a);   // transmittance in front of this Gaussian
    const float wgt = a * T[k];
    const float diff = color_dot(k, cc) - S[k];
    col[0] = wgt * dI[k][0];
    col[1] = col[2] = 0.f;
    if (C == 3) {
      col[1] = wgt * dI[k][1];
      col[2] = wgt * dI[k][2];
    }
    S[k] = fmaf(a, diff, S[k]);   // B <- a c + (1 - a) B
    const float da = diff * T[k];
    const bool uncapped = __fmul_rn(ow, e) < bp.alpha_max;
    dO = uncapped ? e * da : 0.f;
    daa = uncapped ? da * a : 0.f;
    return true;
  };
  // the same for a grid point of a layer whose colour projection cc . dI is
  // ccd: the colour gradient of the layer is the sum of the weights a T
  // (wsum) times dI, formed once per layer (the walk counts its evaluations
  // per row)
  auto adjoint_layer = [&](int k, float a, float e, float ow, float ccd, float& wsum, float& dO) {
    if (a < bp.alpha_min) return false;
    T[k] = __fdividef(T[k], 1.f - a);
    wsum = fmaf(a, T[k], wsum);
    const float diff = ccd - S[k];
    S[k] = fmaf(a, diff, S[k]);
    dO = __fmul_rn(ow, e) < bp.alpha_max ? e * (diff * T[k]) : 0.f;
    return true;
  };
  // the same without branches for a staged point (o = ow): a point below
  // alpha_min (or not listed, o <= 0) leaves T, wsum and S as they are and
  // returns a zero gradient
  auto adjoint_point = [&](int k, float a, float e, float ow, float ccd, float& wsum) {
    const bool ok = ow > 0.f && a >= bp.alpha_min;
    const float Tn = __fdividef(T[k], 1.f - a);
    T[k] = ok ? Tn : T[k];
    const float ae = ok ? a : 0.f;
    wsum = fmaf(ae, T[k], wsum);
    const float diff = ccd - S[k];
    S[k] = fmaf(ae, diff, S[k]);
    return ok && __fmul_rn(ow, e) < bp.alpha_max ? e * (diff * T[k]) : 0.f;
  };
  auto adjoint = [&](int k, float fy, const float4& q, const float4& cc, float& dO, float col[3], float& daa,
                     float& dx, float& dy, float& d2) {
    float e;
    const float a = gauss_alpha(fx, fy, q, bp.alpha_max, dx, dy, d2, e);
    return adjoint_alpha(k, a, e, q.w, cc, dO, col, daa);
  };
  int cur = 0;   // the buffer holding the current staged entry's region
  for (int base = ((wmax - 1) >> 5) << 5; base >= 0 && wmax > 0; base -= 32) {
    const int j = base + lane;
    bool hit = false;
    if (j < wmax) {
      const uint32_t g = gid[rg.x + j];
      const uint32_t gi = g & ~kLayerBit;
      if (g & kLayerBit) {
        const int c = gcurve[gi];
        int4 reg;
        float4 win, loc, org;
        layer_prepare(la, c, tx, ty, wr, reg, win, loc, org);
        hit = reg.x <= reg.y;
        if (hit) {
          s_id[w][lane] = g;
          s_c[w][lane] = color[c];
          s_q[w][lane] = loc;
          s_win[w][lane] = win;
          s_org[w][lane] = org;
          s_rg[w][lane] = reg;
          s_isig[w][lane] = __int_as_float(c);
        }
      } else {
        const float4 q = prep[gi];
        const float2 rs = reach[gi];
        hit = rect_d2(q.x, q.y, wr.x, wr.y, wr.z, wr.w) <= rs.x;
        if (hit) {
          s_q[w][lane] = q;
          s_c[w][lane] = color[gcurve[gi]];
          s_isig[w][lane] = rs.y;
          s_id[w][lane] = g;
        }
      }
    }
    unsigned int mask = __ballot_sync(0xffffffffu, hit);
    __syncwarp();
    // the first staged layer entry's region is requested now; each staged
    // entry requests the next one's before its own walk (every hit entry is
    // walked: wmax bounds the batch)
    if (!per_pair) {
      const int nb = next_staged_layer<kPts, true>(mask, s_id[w], s_rg[w]);
      if (nb >= 0) layer_request<kPts / 32>(la, Gset, s_id[w], s_rg[w], s_q[w], s_org[w], nb, s_pt[w][cur]);
    }
    while (mask) {
      const int b = 31 - __clz(mask);
      mask &= ~(1u << b);
      const int jpos = base + b;
      const uint32_t id = s_id[w][b];
      const float4 cc = s_c[w][b];
      if (id & kLayerBit) {
        bool want[PPT], any = false;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          want[k] = jpos < last[k];
          any = any || want[k];
        }
        if (!__any_sync(0xffffffffu, any)) {   // no pixel of the warp walks this far back
          const int4 r = s_rg[w][b];
          if (!per_pair && (long long)(r.y - r.x + 1) * (r.w - r.z + 1) <= kPts) {
            // its region was requested: pass the request on to the next entry
            cp_async_wait_all();
            __syncwarp();
            const int nb = next_staged_layer<kPts, true>(mask, s_id[w], s_rg[w]);
            if (nb >= 0) layer_request<kPts / 32>(la, Gset, s_id[w], s_rg[w], s_q[w], s_org[w], nb, s_pt[w][cur ^ 1]);
            cur ^= 1;
          }
          continue;
        }
        const uint32_t g0 = id & ~kLayerBit;
        const int c = __float_as_int(s_isig[w][b]);
        const int4 reg = s_rg[w][b];
        const LayerView v = layer_unpack(reg, s_win[w][b], s_q[w][b], s_org[w][b], g0, Gset);
        const float fxl = __fsub_rn(fx, v.X0);
        const int rx0 = reg.x, ry0 = reg.z;
        const int rw = reg.y - reg.x + 1, rh = reg.w - reg.z + 1;
        const bool staged = !per_pair && (long long)rw * rh <= kPts;
        // the region's opacity gradients in s_reg: row r at r rs + a_r, a_r
        // the row's first Gaussian index mod 4, so that an aligned float4 of
        // s_reg holds 4 consecutive Gaussians (quads) when that fits, else
        // packed rows (rs = rw, a_r = 0)
        const int rs_q = (rw + 6) & ~3;
        const bool quads = staged && la.dop != nullptr && rh * rs_q <= kPts;
        const int rs = quads ? rs_q : rw;
        if (staged) {
          cp_async_wait_all();
          __syncwarp();
          const int nb = next_staged_layer<kPts, true>(mask, s_id[w], s_rg[w]);
          if (nb >= 0) layer_request<kPts / 32>(la, Gset, s_id[w], s_rg[w], s_q[w], s_org[w], nb, s_pt[w][cur ^ 1]);
          if (!layer_live<kPts / 32>(s_pt[w][cur], rw * rh, bp.alpha_min)) {
            cur ^= 1;
            continue;
          }
        }
        float csum[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (!want[k]) continue;
          const float fy = py0 + 4 * k + 0.5f;
          const float fyl = __fsub_rn(fy, v.Y0);
          const int sstart = (jpos == last[k] - 1) ? lsub[k] - 1 : 0x7fffffff;
          int ix0, ix1, iy0, iy1;
          layer_window(v, fx, fy, ix0, ix1, iy0, iy1);
          if (staged) {
            const float ccd = color_dot(k, cc);
            float wsum = 0.f;
            for (int iy = iy1; iy >= iy0; --iy) {
              const int rowsub = iy * v.nx;
              const float2* prow = &s_pt[w][cur][(iy - ry0) * rw - rx0];
              float* rreg = &s_reg[w][(iy - ry0) * rs + (quads ? int((g0 + uint32_t(rowsub + rx0)) & 3u) : 0) - rx0];
              const float dy = layer_dy(v, fyl, iy), dy2 = __fmul_rn(dy, dy);
              // the last layer of the pixel starts at its last composited point
              int ix = min(ix1, sstart - rowsub);
              const int ix_start = ix;
              // two points per step: both alphas first, then the adjoint in order
              for (; ix - 1 >= ix0; ix -= 2) {
                const float2 qa = prow[ix], qb = prow[ix - 1];
                float dxa, d2a, ea, dxb, d2b, eb;
                const float aa = layer_alpha_o(v, fxl, dy2, qa, bp.alpha_max, dxa, d2a, ea);
                const float ab = layer_alpha_o(v, fxl, dy2, qb, bp.alpha_max, dxb, d2b, eb);
                const float dOa = adjoint_point(k, aa, ea, qa.y, ccd, wsum);
                if (dOa != 0.f) atomicAdd(&rreg[ix], dOa);
                const float dOb = adjoint_point(k, ab, eb, qb.y, ccd, wsum);
                if (dOb != 0.f) atomicAdd(&rreg[ix - 1], dOb);
              }
              evals += ix_start - ix;   // points whose alpha the loop formed
              if (ix == ix0) {
                const float2 q = prow[ix];
                float dx, d2, e;
                ++evals;
                const float dO = adjoint_point(k, layer_alpha_o(v, fxl, dy2, q, bp.alpha_max, dx, d2, e), e, q.y, ccd, wsum);
                if (dO != 0.f) atomicAdd(&rreg[ix], dO);
              }
            }
            csum[0] = fmaf(wsum, dI[k][0], csum[0]);
            csum[1] = fmaf(wsum, dI[k][1], csum[1]);
            csum[2] = fmaf(wsum, dI[k][2], csum[2]);
            continue;
          }
          for (int iy = iy1; iy >= iy0; --iy) {
            const int rowsub = iy * v.nx;
            const float dy = layer_dy(v, fyl, iy), dy2 = __fmul_rn(dy, dy);
            for (int ix = ix1; ix >= ix0; --ix) {
              if (rowsub + ix > sstart) continue;
              const long long g = v.g_off + rowsub + ix;
              if (g >= v.G) continue;
              const float o = la.rec[g].w;
              if (!layer_o_binned(o, bp.alpha_min)) continue;
              float dO, col[3], daa, dx, d2, e;
              if (!adjoint_alpha(k, layer_alpha_o(v, fxl, dy2, make_float2(layer_qx(v, ix), o), bp.alpha_max, dx, d2,
                                                  e),
                                 e, o, cc, dO, col, daa))
                continue;
              if (!per_pair) {
                csum[0] += col[0];
                csum[1] += col[1];
                csum[2] += col[2];
                if (dO != 0.f) atomicAdd(layer_dop(la, dgauss, g, kRow), dO);
              } else {
                if (full_grads && daa != 0.f) {
                  const float isg = 1.f / la.rec[g].z;
                  const float aa = daa * isg * isg;
                  red_add_v4(dgauss + g * kRow, aa * dx, aa * dy, aa * d2 * isg, 0.f);
                }
                red_add_v4(dgauss + g * kRow + 4, dO, col[0], col[1], col[2]);
              }
            }
          }
        }
        if (!per_pair) {
          // the layer's colour gradient: value k of the warp total sits in lane 8k
          const float cv4[4] = {csum[0], csum[1], csum[2], 0.f};
          const float t0 = warp_sum4(cv4);
          const float t1 = __shfl_down_sync(0xffffffffu, t0, 8);
          const float t2 = __shfl_down_sync(0xffffffffu, t0, 16);
          if (lane == 0 && (t0 != 0.f || t1 != 0.f || t2 != 0.f))
            red_add_v4(dcurve + 4 * (long long)c, t0, t1, t2, 0.f);
        }
        if (staged) {
          __syncwarp();
          if (quads) {
            // one vector reduction per quad of consecutive Gaussians (adding
            // zeros for the padding: other tiles' points, or none)
            const int qr = rs >> 2;
            const float inv_qr = __fdividef(1.f, float(qr));   // the quotients below stay 0.5/qr off integers
            for (int i = lane; i < rh * qr; i += 32) {
              const int r = int((float(i) + 0.5f) * inv_qr);   // exact for the region sizes staged here
              const int jq = i - r * qr;
              float4* sp = reinterpret_cast<float4*>(&s_reg[w][r * rs + 4 * jq]);
              const float4 val = *sp;
              if (val.x != 0.f || val.y != 0.f || val.z != 0.f || val.w != 0.f) {
                *sp = make_float4(0.f, 0.f, 0.f, 0.f);
                const long long gq = ((v.g_off + (long long)(ry0 + r) * v.nx + rx0) & ~3LL) + 4 * jq;
                if (gq + 4 <= la.gcap) {
                  red_add_v4(la.dop + gq, val.x, val.y, val.z, val.w);
                } else {
                  const float vq[4] = {val.x, val.y, val.z, val.w};
#pragma unroll
                  for (int e = 0; e < 4; ++e)
                    if (vq[e] != 0.f && gq + e < la.gcap) atomicAdd(la.dop + gq + e, vq[e]);
                }
              }
            }
          } else {
            const float inv_rw = __fdividef(1.f, float(rw));   // the quotients below stay 0.5/rw off integers
            for (int i = lane; i < rw * rh; i += 32) {
              const float val = s_reg[w][i];
              if (val != 0.f) {
                s_reg[w][i] = 0.f;
                const int iyr = int((float(i) + 0.5f) * inv_rw);
                const int ixr = i - iyr * rw;
                atomicAdd(layer_dop(la, dgauss, v.g_off + (long long)(ry0 + iyr) * v.nx + rx0 + ixr, kRow), val);
              }
            }
          }
          __syncwarp();
          cur ^= 1;
        }
      } else {
        const float4 q = s_q[w][b];
        const float isg_raw = s_isig[w][b];
        const bool geo = full_grads || isg_raw > 0.f;
        const float isg = fabsf(isg_raw);
        float vv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool contrib = false;
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (jpos >= last[k]) continue;
          float dO, col[3], daa, dx, dy, d2;
          if (!adjoint(k, py0 + 4 * k + 0.5f, q, cc, dO, col, daa, dx, dy, d2)) continue;
          contrib = true;
          vv[4] += dO;
          vv[5] += col[0];
          vv[6] += col[1];
          vv[7] += col[2];
          if (geo) {
            const float aa = daa * isg * isg;   // dalpha/dmu = alpha (x - mu) / sigma^2
            vv[0] += aa * dx;
            vv[1] += aa * dy;
            vv[2] += aa * d2 * isg;              // dalpha/dsigma = alpha d^2 / sigma^3
          }
        }
        if (__any_sync(0xffffffffu, contrib)) {
          const uint32_t gg = id & ~kLayerBit;
          if (geo) {
            const float tt = warp_sum8(vv);
            const float t1 = __shfl_down_sync(0xffffffffu, tt, 4);
            const float t2 = __shfl_down_sync(0xffffffffu, tt, 8);
            const float t3 = __shfl_down_sync(0xffffffffu, tt, 12);
            if ((lane & 15) == 0) red_add_v4(dgauss + (long long)gg * kRow + (lane >> 2), tt, t1, t2, t3);
          } else {
            const float tt = warp_sum4(vv + 4);
            const float t1 = __shfl_down_sync(0xffffffffu, tt, 8);
            const float t2 = __shfl_down_sync(0xffffffffu, tt, 16);
            const float t3 = __shfl_down_sync(0xffffffffu, tt, 24);
            if (lane == 0) red_add_v4(dgauss + (long long)gg * kRow + 4, tt, t1, t2, t3);
          }
        }
      }
    }
    cp_async_wait_all();
    __syncwarp();
  }
  count_evals(&st->blend_bwd_evals, evals);
}

// Layer kernels exist for blocks of at most 8 warps (the per-warp regions
// live in static shared memory): tiles 8 and 16, and tile 32 with 4 pixels
// per thread.
static int layer_ppt(int tile, int code) {
  const int ppt = code & ~NS_BLEND_LANE_GROUPS;
  if (tile == 32) return 4;
  if (tile == 8) return ppt >= 2 ? 2 : 1;
  return ppt == 4 ? 4 : (ppt == 2 ? 2 : 1);
}

template <int C>
static void launch_fwd_layers(int tile, int ppt, int grid, cudaStream_t s, const int2* ranges, const uint32_t* gid,
                              const float4* prep, const float2* reach, const int* gcurve, const float4* col,
                              const BlendParams& bp, const LayerArgs& la, float* image, float* Tf, int* nl,
                              DevState* st) {
#define NS_FWDL(TL, PP)                                                                                   \
  do {                                                                                                    \
    static bool carveout = false;                                                                         \
    if (!carveout) {                                                                                      \
      cudaFuncSetAttribute(k_blend_fwd_layers<TL, PP, C>, cudaFuncAttributePreferredSharedMemoryCarveout,  \
                           int(cudaSharedmemCarveoutMaxShared));                                          \
      carveout = true;                                                                                    \
    }                                                                                                     \
    NS_LAUNCH(NS_KERNEL_BLEND_FWD, (k_blend_fwd_layers<TL, PP, C>), grid, (BlendGeom<TL, PP>::kThreads), 0, \
              s, ranges, gid, prep, reach, gcurve, col, bp, la, image, Tf, nl, st);                       \
  } while (0)
  if (tile == 8) { if (ppt == 1) NS_FWDL(8, 1); else NS_FWDL(8, 2); }
  else if (tile == 16) { if (ppt == 1) NS_FWDL(16, 1); else if (ppt == 2) NS_FWDL(16, 2); else NS_FWDL(16, 4); }
  else NS_FWDL(32, 4);
#undef NS_FWDL
}

template <int C>
static void launch_bwd_layers(int tile, int ppt, int grid, cudaStream_t s, const int2* ranges, const uint32_t* gid,
                              const float4* prep, const float2* reach, const int* gcurve, const float4* col,
                              const BlendParams& bp, const LayerArgs& la, const float* dimage, const float* Tf,
                              const int* nl, float* dgauss, DevState* st, int full_grads, float* dcurve) {
  // the register-limited 16 blocks per SM need most of the SM's shared memory
  // (staged regions): ask for the largest carveout once per instantiation
#define NS_BWDL(TL, PP)                                                                                   \
  do {                                                                                                    \
    static bool carveout = false;                                                                         \
    if (!carveout) {                                                                                      \
      cudaFuncSetAttribute(k_blend_bwd_layers<TL, PP, C>, cudaFuncAttributePreferredSharedMemoryCarveout,  \
                           int(cudaSharedmemCarveoutMaxShared));                                          \
      carveout = true;                                                                                    \
    }                                                                                                     \
    NS_LAUNCH(NS_KERNEL_BLEND_BWD, (k_blend_bwd_layers<TL, PP, C>), grid, (BlendGeom<TL, PP>::kThreads), 0, \
              s, ranges, gid, prep, reach, gcurve, col, bp, la, dimage, Tf, nl, dgauss, st, full_grads, dcurve); \
  } while (0)
  if (tile == 8) { if (ppt == 1) NS_BWDL(8, 1); else NS_BWDL(8, 2); }
  else if (tile == 16) { if (ppt == 1) NS_BWDL(16, 1); else if (ppt == 2) NS_BWDL(16, 2); else NS_BWDL(16, 4); }
  else NS_BWDL(32, 4);
#undef NS_BWDL
}

// Kernel of a decomposition: whole-warp sub-blocks, or lane groups (PPT 1-2).
template <int TL, int PP, int C, bool ANISO, bool GRP>
static auto fwd_kernel() {
  if constexpr (GRP && PP <= 2) return &k_blend_fwd_groups<TL, PP, C, ANISO>;
  else return &k_blend_fwd<TL, PP, C, ANISO>;
}
template <int TL, int PP, int C, bool ANISO, bool GRP>
static auto bwd_kernel() {
  if constexpr (GRP && PP <= 2) return &k_blend_bwd_groups<TL, PP, C, ANISO>;
  else return &k_blend_bwd<TL, PP, C, ANISO>;
}

// `code` is a decomposition: pixels per thread, plus NS_BLEND_LANE_GROUPS for
// the lane-group kernels.
template <int C, bool ANISO>
static void launch_fwd(int tile, int code, int grid, cudaStream_t s, const int2* ranges, const uint32_t* gid,
                       const float4* prep, const float2* prep2, const float2* reach, const int* gcurve,
                       const float4* col, const BlendParams& bp, float* image, float* Tf, int* nl, DevState* st) {
  const bool grp = (code & NS_BLEND_LANE_GROUPS) != 0;
  const int ppt = code & ~NS_BLEND_LANE_GROUPS;
#define NS_FWD(TL, PP)                                                                                 \
  {                                                                                                      \
    auto kern = grp ? fwd_kernel<TL, PP, C, ANISO, true>() : fwd_kernel<TL, PP, C, ANISO, false>();      \
    NS_LAUNCH(NS_KERNEL_BLEND_FWD, kern, grid, (BlendGeom<TL, PP>::kThreads), 0, s, ranges, gid, prep,  \
              prep2, reach, gcurve, col, bp, image, Tf, nl, st);                                        \
  }
  if (tile == 8) { if (ppt == 1) NS_FWD(8, 1) else NS_FWD(8, 2) }
  else if (tile == 16) { if (ppt == 1) NS_FWD(16, 1) else if (ppt == 2) NS_FWD(16, 2) else NS_FWD(16, 4) }
  else { if (ppt == 1) NS_FWD(32, 1) else if (ppt == 2) NS_FWD(32, 2) else NS_FWD(32, 4) }
#undef NS_FWD
}

template <int C, bool ANISO>
static void launch_bwd(int tile, int code, int grid, cudaStream_t s, const int2* ranges, const uint32_t* gid,
                       const float4* prep, const float2* prep2, const float2* reach, const int* gcurve,
                       const float4* col, const BlendParams& bp, const float* dimage, const float* Tf, const int* nl,
                       float* dgauss, DevState* st, int full_grads, float* dcurve) {
  const bool grp = (code & NS_BLEND_LANE_GROUPS) != 0;
  const int ppt = code & ~NS_BLEND_LANE_GROUPS;
#define NS_BWD(TL, PP)                                                                                 \
  {                                                                                                      \
    auto kern = grp ? bwd_kernel<TL, PP, C, ANISO, true>() : bwd_kernel<TL, PP, C, ANISO, false>();      \
    NS_LAUNCH(NS_KERNEL_BLEND_BWD, kern, grid, (BlendGeom<TL, PP>::kThreads), 0, s, ranges, gid, prep,  \
              prep2, reach, gcurve, col, bp, dimage, Tf, nl, dgauss, st, full_grads, dcurve);           \
  }
  if (tile == 8) { if (ppt == 1) NS_BWD(8, 1) else NS_BWD(8, 2) }
  else if (tile == 16) { if (ppt == 1) NS_BWD(16, 1) else if (ppt == 2) NS_BWD(16, 2) else NS_BWD(16, 4) }
  else { if (ppt == 1) NS_BWD(32, 1) else if (ppt == 2) NS_BWD(32, 2) else NS_BWD(32, 4) }
#undef NS_BWD
}

// Runtime (channels, tangent-aligned) -> template.
struct BlendArgs {
  const int2* ranges;
  const uint32_t* gid;
  const float4* prep;
  const float2* prep2;
  const float2* reach;
  const int* gcurve;
  const float4* col;
  BlendParams bp;
  float* Tf;
  int* nl;
  DevState* st;
  bool layers;    // fill layers (isotropic sets only)
  LayerArgs la;
};

static void dispatch_fwd(int C, bool aniso, int tile, int ppt, int grid, cudaStream_t s, const BlendArgs& a,
                         float* image) {
  if (a.layers) {
    const int lp = layer_ppt(tile, ppt);
    if (C == 3) launch_fwd_layers<3>(tile, lp, grid, s, a.ranges, a.gid, a.prep, a.reach, a.gcurve, a.col, a.bp, a.la, image, a.Tf, a.nl, a.st);
    else launch_fwd_layers<1>(tile, lp, grid, s, a.ranges, a.gid, a.prep, a.reach, a.gcurve, a.col, a.bp, a.la, image, a.Tf, a.nl, a.st);
    return;
  }
  if (C == 3) {
    if (aniso) launch_fwd<3, true>(tile, ppt, grid, s, a.ranges, a.gid, a.prep, a.prep2, a.reach, a.gcurve, a.col, a.bp, image, a.Tf, a.nl, a.st);
    else launch_fwd<3, false>(tile, ppt, grid, s, a.ranges, a.gid, a.prep, a.prep2, a.reach, a.gcurve, a.col, a.bp, image, a.Tf, a.nl, a.st);
  } else {
    if (aniso) launch_fwd<1, true>(tile, ppt, grid, s, a.ranges, a.gid, a.prep, a.prep2, a.reach, a.gcurve, a.col, a.bp, image, a.Tf, a.nl, a.st);
    else launch_fwd<1, false>(tile, ppt, grid, s, a.ranges, a.gid, a.prep, a.prep2, a.reach, a.gcurve, a.col, a.bp, image, a.Tf, a.nl, a.st);
  }
}

static void dispatch_bwd(int C, bool aniso, int tile, int ppt, int grid, cudaStream_t s, const BlendArgs& a,
                         const float* dimage, float* dgauss, int full_grads, float* dcurve) {
  if (a.layers) {
    const int lp = layer_ppt(tile, ppt);
    if (C == 3) launch_bwd_layers<3>(tile, lp, grid, s, a.ranges, a.gid, a.prep, a.reach, a.gcurve, a.col, a.bp, a.la, dimage, a.Tf, a.nl, dgauss, a.st, full_grads, dcurve);
    else launch_bwd_layers<1>(tile, lp, grid, s, a.ranges, a.gid, a.prep, a.reach, a.gcurve, a.col, a.bp, a.la, dimage, a.Tf, a.nl, dgauss, a.st, full_grads, dcurve);
    return;
  }
  if (C == 3) {
    if (aniso) launch_bwd<3, true>(tile, ppt, grid, s, a.ranges, a.gid, a.prep, a.prep2, a.reach, a.gcurve, a.col, a.bp, dimage, a.Tf, a.nl, dgauss, a.st, full_grads, dcurve);
    else launch_bwd<3, false>(tile, ppt, grid, s, a.ranges, a.gid, a.prep, a.prep2, a.reach, a.gcurve, a.col, a.bp, dimage, a.Tf, a.nl, dgauss, a.st, full_grads, dcurve);
  } else {
    if (aniso) launch_bwd<1, true>(tile, ppt, grid, s, a.ranges, a.gid, a.prep, a.prep2, a.reach, a.gcurve, a.col, a.bp, dimage, a.Tf, a.nl, dgauss, a.st, full_grads, dcurve);
    else launch_bwd<1, false>(tile, ppt, grid, s, a.ranges, a.gid, a.prep, a.prep2, a.reach, a.gcurve, a.col, a.bp, dimage, a.Tf, a.nl, dgauss, a.st, full_grads, dcurve);
  }
}

// ---------------------------------------------------------------------------

struct RasterPlan {
  int passes, bits_per_pass;
};

static RasterPlan radix_plan(int n_tiles) {
  int bits = 1;
  while ((1LL << bits) < n_tiles) ++bits;
  RasterPlan r;
  r.passes = (bits + 7) / 8;
  r.bits_per_pass = (bits + r.passes - 1) / r.passes;
  return r;
}

static BlendParams blend_params(const Layout& L, const ns_raster_params* rp) {
  BlendParams bp;
  bp.alpha_min = rp->alpha_min;
  bp.alpha_max = rp->alpha_max;
  bp.t_min = rp->t_min;
  bp.bg0 = rp->bg[0];
  bp.bg1 = rp->bg[1];
  bp.bg2 = rp->bg[2];
  bp.W = L.W;
  bp.H = L.H;
  bp.tiles_x = L.tiles_x;
  bp.tiles_per_scene = L.tiles_x * L.tiles_y;
  return bp;
}

// Whether a Gaussian set is binned by fill layers, and what the layer kernels read.
static bool use_layers(const ns_raster_params* rp, const ns_gaussians* g) {
  return rp->fill_layers != 0 && g->shape == nullptr;
}

static LayerArgs layer_args(const Layout& L, const ns_raster_params* rp, const ns_gaussians* g, void* ws) {
  LayerArgs la;
  la.plan = at<CurvePlan>(ws, L.o_plan);
  la.rec = reinterpret_cast<const float4*>(g->rec);
  la.gcount = g->count;
  la.gcap = int(L.gcap);
  la.tile = rp->tile;
  la.k_sigma = rp->k_sigma;
  la.inv_tile = 1.f / float(rp->tile);
  la.log_amin = rp->alpha_min > 0.f ? logf(rp->alpha_min) : -INFINITY;
  la.nsub = at<int>(ws, L.o_nsub);
  la.runs = at<int2>(ws, L.o_lruns);
  la.lconst = at<float4>(ws, L.o_lconst);
  la.tiles_x = L.tiles_x;
  la.runs_stride = L.tiles_x + L.tiles_y;
  la.dop = nullptr;
  return la;
}

static int resolve_ppt(int tile, int ppt) {
  if (ppt == 0) return tile == 8 ? 1 : 2;   // library default
  return ppt;
}

static bool ppt_ok(int tile, int code) {
  const int ppt = code & ~NS_BLEND_LANE_GROUPS;
  if (code & NS_BLEND_LANE_GROUPS) return ppt == 1 || ppt == 2;
  return ppt == 1 || ppt == 2 || (ppt == 4 && tile >= 16);
}

static bool check_raster(const ns_raster_params* rp) {
  if (!rp || (rp->tile != 8 && rp->tile != 16 && rp->tile != 32) || !(rp->k_sigma > 0.f) ||
      !(rp->alpha_max > 0.f) || !(rp->alpha_max < 1.f) || !(rp->alpha_min >= 0.f) || !(rp->t_min >= 0.f) ||
      !(rp->t_min < 1.f)) {
    set_error("invalid raster parameters (tile 8, 16 or 32; 0 < alpha_max < 1; k_sigma > 0)");
    return false;
  }
  if (!ppt_ok(rp->tile, resolve_ppt(rp->tile, rp->ppt_fwd)) || !ppt_ok(rp->tile, resolve_ppt(rp->tile, rp->ppt_bwd))) {
    set_error("invalid blend decomposition (pixels per thread 1, 2, or 4 with tiles of 16 and 32; "
              "lane groups with 1 or 2; 0 = default)");
    return false;
  }
  return true;
}

// Sorted-pair buffer index after the sort (for tools).
int sorted_buffer(const Layout& L) { return radix_plan(L.n_tiles).passes & 1; }

}  // namespace ns

using namespace ns;

extern "C" ns_status splat_forward(const ns_curves* curves, const ns_gaussians* g, const ns_raster_params* rp,
                                   const ns_capacity* cap, float* image, void* ws, size_t ws_bytes, void* stream) {
  Layout L;
  if (!curves || !g || !cap || !image || !ws || !g->rec || !g->curve || !g->count) {
    set_error("splat_forward: null argument");
    return NS_ERR_INVALID_ARG;
  }
  if (!check_raster(rp)) return NS_ERR_INVALID_ARG;
  if (!make_layout(curves, cap, rp, &L)) return NS_ERR_INVALID_ARG;
  if (ws_bytes < L.total || g->capacity < cap->gaussians) {
    set_error("splat_forward: workspace or Gaussian arrays smaller than the capacities");
    return NS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevState* st = at<DevState>(ws, L.o_state);
  int* curve_scene = at<int>(ws, L.o_curve_scene);
  int* bsum = at<int>(ws, L.o_bsum);
  uint32_t* k0 = at<uint32_t>(ws, L.o_k0);
  uint32_t* v0 = at<uint32_t>(ws, L.o_v0);
  uint32_t* k1 = at<uint32_t>(ws, L.o_k1);
  uint32_t* v1 = at<uint32_t>(ws, L.o_v1);
  uint32_t* hist = at<uint32_t>(ws, L.o_hist);
  uint32_t* totals = hist + 256 * (size_t)L.sort_blocks;   // 256 per radix pass, after the histogram
  int2* ranges = at<int2>(ws, L.o_ranges);
  float* Tf = at<float>(ws, L.o_T);
  int* nl = at<int>(ws, L.o_nlast);
  const float4* rec = reinterpret_cast<const float4*>(g->rec);

  BinParams bp;
  bp.k_sigma = rp->k_sigma;
  bp.inv_tile = 1.f / float(rp->tile);
  bp.alpha_min = rp->alpha_min;
  bp.log_amin = rp->alpha_min > 0.f ? logf(rp->alpha_min) : -INFINITY;
  bp.tiles_x = L.tiles_x;
  bp.tiles_y = L.tiles_y;
  bp.tiles_per_scene = L.tiles_x * L.tiles_y;
  bp.n_curves = L.nc;
  bp.gcap = int(L.gcap);
  bp.fill_layers = use_layers(rp, g) ? 1 : 0;
  bp.lmin = at<int2>(ws, L.o_lmin);
  bp.lmax = at<int2>(ws, L.o_lmax);
  bp.lbox = at<const int4>(ws, L.o_lbox);
  bp.bmix = at<const int>(ws, L.o_bmix);
  bp.bflag = at<int>(ws, L.o_bflag);
  bp.lcount = at<int>(ws, L.o_lcount);
  const CurvePlan* plan = at<CurvePlan>(ws, L.o_plan);
  {
    // curve scenes, counters, tile ranges and layer extremes in one launch
    const int want = std::max((curves->n_curves + 255) / 256, std::min((L.n_tiles + 2047) / 2048, num_sms()));
    NS_LAUNCH(NS_KERNEL_OTHER, k_curve_scene, std::max(1, want), 256, 0, s, *curves, curve_scene, st, ranges,
              L.n_tiles, bp.fill_layers ? bp.lmin : nullptr, bp.lmax);
  }
  const int bin_blocks = int(L.bin_blocks);
  const bool aniso = g->shape != nullptr;
  const float4* shape = reinterpret_cast<const float4*>(g->shape);
  if (bin_blocks > 0) {
    auto kc = aniso ? &k_bin_count<true> : &k_bin_count<false>;
    NS_LAUNCH(NS_KERNEL_BIN_COUNT, kc, int(std::min<long long>(bin_blocks, num_sms() * 8LL)), 256, 0, s, rec, shape, g->curve, curves->flags, g->count, bp, bsum, st,
              at<float4>(ws, L.o_prep), at<float2>(ws, L.o_prep2), at<float2>(ws, L.o_reach), plan);
  }
  if (bp.fill_layers && L.nc > 0 && bin_blocks > 0)
    NS_LAUNCH(NS_KERNEL_OTHER, k_layer_count, (L.nc + 127) / 128, 128, 0, s, *curves, plan, rec, g->count, bp, bsum,
              st);
  NS_LAUNCH(NS_KERNEL_SCAN, k_scan_small, 1, 1024, 0, s, bsum, g->count, int(L.gcap), kBinItems, st, cap->pairs,
            totals, 256 * kMaxRadixPasses);
  if (bp.fill_layers && L.nc > 0 && bin_blocks > 0)
    NS_LAUNCH(NS_KERNEL_OTHER, k_layer_emit, L.nc, 128, 0, s, *curves, plan, rec, g->count,
              curve_scene, bp, bsum, at<const int>(ws, L.o_order), k0, v0, cap->pairs, st);
  if (bin_blocks > 0) {
    auto ke = aniso ? &k_bin_emit<true> : &k_bin_emit<false>;
    NS_LAUNCH(NS_KERNEL_BIN_EMIT, ke, int(std::min<long long>(bin_blocks, num_sms() * 8LL)), 256, 0, s, rec, shape, g->curve, g->count, curve_scene, bp, bsum,
              k0, v0, cap->pairs, curves->flags, plan);
  }
  const RasterPlan rpn = radix_plan(L.n_tiles);
  const int sort_blocks = int(L.sort_blocks);
  const int sort_grid = std::min(sort_blocks, num_sms() * 4);   // the kernels stride over the pairs' blocks
  uint32_t *kin = k0, *vin = v0, *kout = k1, *vout = v1;
  for (int pass = 0; pass < rpn.passes; ++pass) {
    const int shift = pass * rpn.bits_per_pass;
    if (sort_blocks > 0) {
      uint32_t* tot = totals + 256 * pass;
      NS_LAUNCH(NS_KERNEL_RADIX_HIST, k_radix_hist, sort_grid, kSortThreads, 0, s, kin, st, shift,
                rpn.bits_per_pass, hist, tot);
      NS_LAUNCH(NS_KERNEL_SCAN, k_radix_scan, 1 << rpn.bits_per_pass, 256, 0, s, hist, st, tot);
      NS_LAUNCH(NS_KERNEL_RADIX_SCATTER, k_radix_scatter, sort_grid, kSortThreads, 0, s, kin, vin, kout, vout, hist,
                st, shift, rpn.bits_per_pass);
    }
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  if (bp.fill_layers && L.nc > 0)
    NS_LAUNCH(NS_KERNEL_OTHER, k_layer_runs, L.nc, 128, 0, s, *curves, plan, rec, g->count, bp,
              at<int2>(ws, L.o_lruns), L.tiles_x + L.tiles_y, at<float4>(ws, L.o_lconst),
              at<const float2>(ws, L.o_glo));
  NS_LAUNCH(NS_KERNEL_RANGES, k_ranges, num_sms() * 16, 256, 0, s, kin, st, ranges);
  const BlendArgs ba{ranges, vin, at<float4>(ws, L.o_prep), at<float2>(ws, L.o_prep2), at<float2>(ws, L.o_reach),
                     g->curve, reinterpret_cast<const float4*>(curves->color), blend_params(L, rp), Tf, nl, st,
                     use_layers(rp, g), layer_args(L, rp, g, ws)};
  dispatch_fwd(L.C, aniso, rp->tile, resolve_ppt(rp->tile, rp->ppt_fwd), L.n_tiles, s, ba, image);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("splat_forward: ") + cudaGetErrorString(e));
    return NS_ERR_CUDA;
  }
  return NS_OK;
}

namespace ns {
// Blend adjoint, used by splat_backward (ns_backward.cu).  With full_grads = 0
// the caller's per-curve colour gradients `dcurve` ({r, g, b, o} per curve,
// already zeroed or accumulating) may receive the colour gradients of fill
// Gaussians directly instead of their per-Gaussian rows.
bool layers_active(const ns_raster_params* rp, const ns_gaussians* g) { return use_layers(rp, g); }

ns_status launch_blend_bwd(const Layout& L, const ns_curves* curves, const ns_gaussians* g,
                           const ns_raster_params* rp, const float* dimage, float* dgauss, void* ws,
                           cudaStream_t s, int full_grads, float* dcurve, float* dop) {
  const RasterPlan rpn = radix_plan(L.n_tiles);
  const uint32_t* vsorted = (rpn.passes & 1) ? at<uint32_t>(ws, L.o_v1) : at<uint32_t>(ws, L.o_v0);
  DevState* st = at<DevState>(ws, L.o_state);   // its counters were cleared by the caller
  BlendArgs ba{at<int2>(ws, L.o_ranges), vsorted, at<float4>(ws, L.o_prep), at<float2>(ws, L.o_prep2),
               at<float2>(ws, L.o_reach), g->curve, reinterpret_cast<const float4*>(curves->color),
               blend_params(L, rp), at<float>(ws, L.o_T), at<int>(ws, L.o_nlast), st,
               use_layers(rp, g), layer_args(L, rp, g, ws)};
  ba.la.dop = dop;
  dispatch_bwd(L.C, g->shape != nullptr, rp->tile, resolve_ppt(rp->tile, rp->ppt_bwd), L.n_tiles, s, ba, dimage,
               dgauss, full_grads, full_grads ? nullptr : dcurve);
  return NS_OK;
}
bool raster_params_ok(const ns_raster_params* rp) { return check_raster(rp); }
}  // namespace ns

extern "C" ns_status ns_autotune_blend(const ns_curves* curves, const ns_gaussians* g, ns_raster_params* rp,
                                       const ns_capacity* cap, float* image, const float* dL_dimage, void* ws,
                                       size_t ws_bytes, int32_t repeats, void* stream) {
  Layout L;
  if (!curves || !g || !rp || !cap || !image || !ws || repeats < 1) {
    set_error("ns_autotune_blend: null argument or repeats < 1");
    return NS_ERR_INVALID_ARG;
  }
  if (!check_raster(rp) || !make_layout(curves, cap, rp, &L)) return NS_ERR_INVALID_ARG;
  if (ws_bytes < L.total) {
    set_error("ns_autotune_blend: workspace smaller than the layout");
    return NS_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevState* st = at<DevState>(ws, L.o_state);
  const RasterPlan rpn = radix_plan(L.n_tiles);
  const uint32_t* vsorted = (rpn.passes & 1) ? at<uint32_t>(ws, L.o_v1) : at<uint32_t>(ws, L.o_v0);
  float* dg = at<float>(ws, L.o_dgauss);
  const bool aniso = g->shape != nullptr;
  const int row = aniso ? 12 : 8;
  const BlendArgs ba{at<int2>(ws, L.o_ranges), vsorted, at<float4>(ws, L.o_prep), at<float2>(ws, L.o_prep2),
                     at<float2>(ws, L.o_reach), g->curve, reinterpret_cast<const float4*>(curves->color),
                     blend_params(L, rp), at<float>(ws, L.o_T), at<int>(ws, L.o_nlast), st,
                     use_layers(rp, g), layer_args(L, rp, g, ws)};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    set_error("ns_autotune_blend: cudaEventCreate failed");
    return NS_ERR_CUDA;
  }
  auto fwd = [&](int ppt) { dispatch_fwd(L.C, aniso, rp->tile, ppt, L.n_tiles, s, ba, image); };
  // the per-curve colour gradients of the timed adjoint go to the knot-gradient
  // scratch (at least 11 floats per curve; splat_backward clears it before use)
  float* dcurve_scratch = at<float>(ws, L.o_dknots);
  auto bwd = [&](int ppt) {
    dispatch_bwd(L.C, aniso, rp->tile, ppt, L.n_tiles, s, ba, dL_dimage, dg, 0, dcurve_scratch);
  };
  auto time_best = [&](bool backward) {
    int best = 0;
    float best_ms = 3.4e38f;
    for (int ppt : {1, 2, 4, 1 | NS_BLEND_LANE_GROUPS, 2 | NS_BLEND_LANE_GROUPS}) {
      if (!ppt_ok(rp->tile, ppt) && !(ba.layers && ppt == 4)) continue;
      if (ba.layers && layer_ppt(rp->tile, ppt) != ppt) continue;   // the layer kernels' own settings
      float t = 3.4e38f;
      for (int r = 0; r < repeats + 1; ++r) {   // the first run warms the variant up
        if (backward) cudaMemsetAsync(dg, 0, sizeof(float) * row * (size_t)L.gcap, s);
        cudaEventRecord(e0, s);
        if (backward) bwd(ppt); else fwd(ppt);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms < t) t = ms;
      }
      if (t < best_ms) {
        best_ms = t;
        best = ppt;
      }
    }
    return best;
  };
  const int bf = time_best(false);
  const int bb = dL_dimage ? time_best(true) : resolve_ppt(rp->tile, rp->ppt_bwd);
  rp->ppt_fwd = bf;
  rp->ppt_bwd = bb;
  // leave the workspace as the chosen forward leaves it (the results of all
  // variants are identical) and the counters as one forward pass sets them
  cudaMemsetAsync(&st->blend_evals, 0, 5 * sizeof(unsigned long long), s);
  fwd(bf);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    set_error(std::string("ns_autotune_blend: ") + cudaGetErrorString(e));
    return NS_ERR_CUDA;
  }
  return NS_OK;
}
