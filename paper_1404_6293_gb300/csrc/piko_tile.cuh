// piko_tile.cuh -- device code of the per-tile Process stage, shared by the
// single-scene kernel (piko_process.cu) and the multi-scene batch kernels
// (piko_batch.cu).
//
// Rasterizer, fragment shader and depth test fused into one stage (the
// kernel fusion of Sec. 5.2.1 of the Piko paper), with the tile's depth|ID
// buffer in shared memory (the on-chip depth buffer Sec. 5.2.4 names).
//
// Per tile:
//  1. each thread takes one bin entry, re-derives the triangle from the
//     snapped vertices and stores what shading needs (edge coordinates, 1/A
//     and the vertex attributes) in a shared-memory record.  A small box
//     inside the tile is walked by the thread for coverage only, and the
//     warp then shares out the covered samples of all its small boxes for
//     their depths (fragment_pass); larger boxes go to a queue that whole
//     warps rasterize 32 pixels at a time with a coverage ballot;
//  2. every covered sample does a 64-bit atomic minimum on the tile's key,
//     key = depth << 40 | triangle << slot_bits | record slot: ordered by
//     (depth, triangle) exactly like depth << 32 | triangle, since a
//     triangle has one record per tile;
//  3. one thread per pixel shades the winner from its record and writes the
//     key (as depth << 32 | triangle) and the colour, rows contiguous.
#pragma once

#include <cuda_fp16.h>

#include "piko_internal.cuh"

namespace piko {

// What the Process stage needs of one scene.  vtx and vdot point at this
// scene's first vertex; bin entries hold triangle indices offset by tri_base.
struct TileScene {
  RasterGeom g;
  int mode, unclamped, small_px;
  int slot_bits, nslots, rec_stride;
  int tri_base;
  const int* tris;
  const int4* vtx;
  const float* color;
  const float* normal;
  const float* light;
  const float* vdot;
  const float* invw;  // 1 / clip w per vertex, or NULL for screen-space attributes
  // near/far clipping: triangles T.. of the frame are clipped sub-triangles
  // (3 snapped points each in clip_tris, their triangle in clip_orig); pos
  // and mvp give a clipped winner's clip coordinates for shading (NULL: no
  // clipping)
  int T;
  const int4* clip_tris;
  const unsigned* clip_orig;
  const float4* pos;
  const float* mvp;
  unsigned long long* key_out;
  float4* rgba_out;
  uint2* gnorm_out;
  uint2* galb_out;
};

// Per-CTA shared memory of the stage.
// Each lane owns FST_WORDS staging words per bin entry, stored word-major
// per warp (word w of lane l at w * 32 + l, so that a lane's words fall in
// its own bank).  A lane uses them for one of two things:
//  - a small box: the triangle's depth setup, read by the warp's
//    fragment_pass (FS_* words);
//  - a large triangle queued for the warps: its snapped vertices, depths and
//    area as set up by the lane that met it (so that the warp re-reads
//    nothing from global memory), then its triangle index and record slot
//    (BG_* words).
// After the staging words, each warp has a list of up to FRAG_CAP fragment
// descriptors.  The queue of large triangles holds the thread index of each.
constexpr int FST_WORDS = 13;
constexpr int FRAG_CAP = 128;
constexpr int FRAG_WARP_WORDS = FST_WORDS * 32 + FRAG_CAP;
enum { BG_X0 = 0, BG_Y0, BG_X1, BG_Y1, BG_X2, BG_Y2, BG_Z0, BG_Z1, BG_Z2, BG_ALO, BG_AHI, BG_T, BG_SLOT };

struct TileSmem {
  unsigned long long* skey;  // [bin_px], all KEY_EMPTY between tiles
  int* sbig;                 // [nt] ring of the threads whose large triangles are queued
  int* sfrag;                // [nt / 32][FRAG_WARP_WORDS]
  int* srec;                 // [nslots][rec_stride]
  unsigned* s_nbig;          // grows monotonically
};

struct TileStats {
  unsigned long long tests, frags, shaded;
};

// record words: 0..5 X0 Y0 X1 Y1 X2 Y2 (oriented), 6 = 1/A (float), then the
// attributes, then (perspective-correct attributes only) 1/w of the three
// vertices
constexpr int R_RA = 6;
constexpr int R_ATTR = 7;

__host__ __device__ __forceinline__ int rec_attr_count(int mode, bool has_color) {
  if (mode == PIKO_SHADE_GOURAUD) return 9;              // c0 c1 c2
  if (mode == PIKO_SHADE_LAMBERT) return has_color ? 12 : 3;  // d0 d1 d2 (n_i . L) [+ c0 c1 c2]
  return 18;                                             // n0 n1 n2 c0 c1 c2
}


// ---------------------------------------------------------------- raster
// Large boxes of at least this many pixels in a tile are walked by row spans
// (raster_warp_spans), smaller ones sample by sample (raster_warp).
#ifndef PIKO_SPAN_MIN_PX
#define PIKO_SPAN_MIN_PX 128
#endif

template <typename I>
struct Edges {
  I e0, e1, e2;     // edge functions minus the fill-rule bias (covered iff all >= 0)
  I sx0, sx1, sx2;  // steps per pixel in x
  I sy0, sy1, sy2;  // steps per pixel in y
  int b1, b2;       // biases of edges 1 and 2
};

template <typename I>
__device__ __forceinline__ Edges<I> make_edges(const TriSetup& s, int px, int py) {
  Edges<I> e;
  const I Px = (I)256 * px + 128, Py = (I)256 * py + 128;
  const int dx0 = s.X2 - s.X1, dy0 = s.Y2 - s.Y1;
  const int dx1 = s.X0 - s.X2, dy1 = s.Y0 - s.Y2;
  const int dx2 = s.X1 - s.X0, dy2 = s.Y1 - s.Y0;
  const int b0 = 1 - top_left(dx0, dy0);
  e.b1 = 1 - top_left(dx1, dy1);
  e.b2 = 1 - top_left(dx2, dy2);
  // coordinate differences are below 2^24 and fit int32
  e.e0 = (I)dx0 * (I)((int)Py - s.Y1) - (I)dy0 * (I)((int)Px - s.X1) - b0;
  e.e1 = (I)dx1 * (I)((int)Py - s.Y2) - (I)dy1 * (I)((int)Px - s.X2) - e.b1;
  e.e2 = (I)dx2 * (I)((int)Py - s.Y0) - (I)dy2 * (I)((int)Px - s.X0) - e.b2;
  e.sx0 = (I)-256 * dy0; e.sx1 = (I)-256 * dy1; e.sx2 = (I)-256 * dy2;
  e.sy0 = (I)256 * dx0;  e.sy1 = (I)256 * dx1;  e.sy2 = (I)256 * dx2;
  return e;
}

__device__ __forceinline__ void key_store(unsigned long long* skey, int idx, unsigned z, unsigned long long tag) {
  const unsigned long long k = ((unsigned long long)z << 40) | tag;
  if (k < skey[idx]) atomicMin(skey + idx, k);
}

// Depth for a covered sample of a triangle with A < 2^31: then w1, w2 >= 0
// and w1 + w2 <= A fit 32 bits, so the quotient is estimated from float32
// barycentrics (32-bit conversions only) and corrected exactly against the
// 64-bit numerator w1 (Z1 - Z0) + w2 (Z2 - Z0).
__device__ __forceinline__ void key_min_mid(unsigned long long* skey, int idx, int w1, int w2, const TriSetup& s,
                                            float rA, unsigned long long tag) {
  const int d1 = s.Z1 - s.Z0, d2 = s.Z2 - s.Z0;
  const int A = (int)s.A;
  int q = __float2int_rd((float)w1 * rA * (float)d1 + (float)w2 * rA * (float)d2);
  long long r = (long long)w1 * d1 + (long long)w2 * d2 - (long long)q * A;
  for (int it = 0; r < 0 && it < DIV_FIX_LIMIT; ++it) { --q; r += A; }
  for (int it = 0; r >= A && it < DIV_FIX_LIMIT; ++it) { ++q; r -= A; }
  key_store(skey, idx, (unsigned)(s.Z0 + q), tag);
}

// Depth keys of the per-thread walk over a small box (bounding box below
// 2^15 in 16.8 units, so A < 2^30).  The quotient q = floor((w1 d1 + w2 d2) / A),
// d_i = Z_i - Z0, is estimated in float32 from k_i = d_i / A (per entry) and
// then corrected against the exact remainder r = w1 d1 + w2 d2 - q A, with
// w1, w2 in [0, A] for a covered sample.  The estimate is within
// (|d1| + |d2|) 2^-21 + 1 of q (1/A to 2 ulp, four roundings), so:
//  - fast (A < 2^27 and |d1| + |d2| < 2^22): |r| < 4A < 2^29, and 32-bit
//    wrapping arithmetic gives r exactly;
//  - otherwise r is formed in 64 bits and the estimate is within 16 of q.
// The choice is per entry, so a warp rarely splits between the two forms.
// The key is Z0 << 40 | tag plus q << 40 (Z0 + q stays in [0, 2^24)).
struct DepthSetup {
  int d1, d2, A;
  float k1, k2;
  unsigned long long kbase;
  bool fast;
};

__device__ __forceinline__ DepthSetup depth_setup(const TriSetup& s, float rA, unsigned long long tag) {
  DepthSetup d;
  d.d1 = s.Z1 - s.Z0;
  d.d2 = s.Z2 - s.Z0;
  d.A = (int)s.A;
  d.k1 = rA * (float)d.d1;
  d.k2 = rA * (float)d.d2;
  d.kbase = ((unsigned long long)(unsigned)s.Z0 << 40) | tag;
  d.fast = s.A < (1LL << 27) && abs(d.d1) + abs(d.d2) < (1 << 22);
  return d;
}

__device__ __forceinline__ void key_min_box(unsigned long long* skey, int idx, int w1, int w2, const DepthSetup& d) {
  int q = __float2int_rd(__fmaf_rn((float)w1, d.k1, (float)w2 * d.k2));
  if (d.fast) {
    int r = (int)((unsigned)w1 * (unsigned)d.d1 + (unsigned)w2 * (unsigned)d.d2 - (unsigned)q * (unsigned)d.A);
    for (int it = 0; r < 0 && it < DIV_FIX_LIMIT; ++it) { --q; r += d.A; }
    for (int it = 0; r >= d.A && it < DIV_FIX_LIMIT; ++it) { ++q; r -= d.A; }
  } else {
    long long r = (long long)w1 * d.d1 + (long long)w2 * d.d2 - (long long)q * d.A;
    for (int it = 0; r < 0 && it < DIV_FIX_LIMIT; ++it) { --q; r += d.A; }
    for (int it = 0; r >= d.A && it < DIV_FIX_LIMIT; ++it) { ++q; r -= d.A; }
  }
  const unsigned long long k = d.kbase + ((unsigned long long)(long long)q << 40);
  if (k < skey[idx]) atomicMin(skey + idx, k);
}

__device__ __forceinline__ void key_min_large(unsigned long long* skey, int idx, long long w1, long long w2,
                                              const TriSetup& s, float rA, unsigned long long tag) {
  key_store(skey, idx, depth_of(w1, w2, s, rA), tag);
}


// One thread walks the box of a small triangle inside the tile.  With I =
// int the triangle's bounding box is below 2^15 in 16.8 units in both
// directions, so every edge value inside the box is below 2^31 in magnitude
// and int32 arithmetic is exact.
template <typename I>
__device__ __forceinline__ unsigned raster_thread_body(const TriSetup& s, unsigned long long tag, int px0, int px1,
                                                       int py0, int py1, int x0, int y0, int bshift_x,
                                                       unsigned long long* skey) {
  const Edges<I> e = make_edges<I>(s, px0, py0);
  const float rA = approx_rcp(f32_from_i64(s.A));
  const DepthSetup d = depth_setup(s, rA, tag);
  unsigned frags = 0;
  I r0 = e.e0, r1 = e.e1, r2 = e.e2;
  // walk by tile-local pixel index: first and one-past-last of each row
  const int bw = px1 - px0 + 1, pitch = 1 << bshift_x;
  const int first = ((py0 - y0) << bshift_x) + (px0 - x0);
  const int last = first + ((py1 - py0) << bshift_x);
  for (int row = first; row <= last; row += pitch) {
    I a0 = r0, a1 = r1, a2 = r2;
    for (int idx = row; idx < row + bw; ++idx) {
      if ((a0 | a1 | a2) >= 0) {
        if (sizeof(I) == 4)
          key_min_box(skey, idx, (int)a1 + e.b1, (int)a2 + e.b2, d);
        else
          key_min_large(skey, idx, (long long)a1 + e.b1, (long long)a2 + e.b2, s, rA, tag);
        ++frags;
      }
      a0 += e.sx0; a1 += e.sx1; a2 += e.sx2;
    }
    r0 += e.sy0; r1 += e.sy1; r2 += e.sy2;
  }
  return frags;
}

// Small boxes of small triangles (the common case) stay inline; the int64
// form for small boxes of large triangles is a separate instance.
__device__ __forceinline__ unsigned raster_thread32(const TriSetup& s, unsigned long long tag, int px0, int px1,
                                                    int py0, int py1, int x0, int y0, int bshift_x,
                                                    unsigned long long* skey) {
  return raster_thread_body<int>(s, tag, px0, px1, py0, py1, x0, y0, bshift_x, skey);
}
__device__ __forceinline__ unsigned raster_thread64(const TriSetup& s, unsigned long long tag, int px0, int px1,
                                                 int py0, int py1, int x0, int y0, int bshift_x,
                                                 unsigned long long* skey) {
  return raster_thread_body<long long>(s, tag, px0, px1, py0, py1, x0, y0, bshift_x, skey);
}

// ------------------------------------------------ compacted small boxes
// A small box (at most 32 pixels, of a triangle whose bounding box is below
// 2^15 in 16.8 units, so that the int32 edge walk is exact) is walked by its
// thread for coverage only, into a mask whose bit j is the box's j-th pixel
// in row-major order.  The lane stores the triangle's depth setup in the
// warp's staging area, and fragment_pass then gives the warp's covered
// samples out to consecutive lanes: the depth quotient, key and shared
// minimum, most of a tile of tiny triangles' work, run with every lane busy
// instead of each lane following its own box.
struct SmallBox {
  unsigned mask;  // covered pixels of the box
  int place;      // tile-local index of the box's first pixel | box width << 16
};

// staging words of a lane (word w of lane l at w * 32 + l)
enum { FS_E1 = 0, FS_E2, FS_SX1, FS_SY1, FS_SX2, FS_SY2, FS_K1, FS_K2, FS_D1, FS_D2, FS_A, FS_KLO, FS_KHI };

__device__ __forceinline__ void small_box(const TriSetup& s, unsigned long long tag, int px0, int px1, int py0,
                                          int py1, int x0, int y0, int bshift_x, int* wst, int lane, SmallBox& b) {
  const Edges<int> e = make_edges<int>(s, px0, py0);
  const int bw = px1 - px0 + 1, bh = py1 - py0 + 1;
  // shift each sample's coverage in from the top; the last sample ends at bit n - 1
  unsigned mask = 0u;
  int r0 = e.e0, r1 = e.e1, r2 = e.e2;
  for (int y = 0; y < bh; ++y) {
    int a0 = r0, a1 = r1, a2 = r2;
    for (int x = 0; x < bw; ++x) {
      mask = (mask >> 1) | (~(unsigned)(a0 | a1 | a2) & 0x80000000u);
      a0 += e.sx0; a1 += e.sx1; a2 += e.sx2;
    }
    r0 += e.sy0; r1 += e.sy1; r2 += e.sy2;
  }
  b.mask = mask >> (32 - bw * bh);
  if (b.mask == 0u) return;
  b.place = (((py0 - y0) << bshift_x) + (px0 - x0)) | (bw << 16);
  const float rA = approx_rcp(f32_from_i64(s.A));
  const DepthSetup d = depth_setup(s, rA, tag);
  int* w = wst + lane;
  w[FS_E1 * 32] = e.e1 + e.b1;  // exact edge functions at the box's first pixel
  w[FS_E2 * 32] = e.e2 + e.b2;
  w[FS_SX1 * 32] = e.sx1; w[FS_SY1 * 32] = e.sy1;
  w[FS_SX2 * 32] = e.sx2; w[FS_SY2 * 32] = e.sy2;
  w[FS_K1 * 32] = __float_as_int(d.k1); w[FS_K2 * 32] = __float_as_int(d.k2);
  w[FS_D1 * 32] = d.d1; w[FS_D2 * 32] = d.d2;
  w[FS_A * 32] = d.fast ? d.A : -d.A;
  w[FS_KLO * 32] = (int)(unsigned)d.kbase;
  w[FS_KHI * 32] = (int)(unsigned)(d.kbase >> 32);
}

// Depth key of one compacted fragment: descriptor = tile-local pixel index
// (12 bits) | column in the box << 12 | row << 17 | staging lane << 22.  The
// same quotient and key as key_min_box.
__device__ __forceinline__ void fragment_key(const int* wst, unsigned desc, unsigned long long* skey) {
  const int* w = wst + (desc >> 22);
  const int rx = (desc >> 12) & 31, ry = (desc >> 17) & 31, idx = desc & 0xFFF;
  // covered: w1, w2 in [0, A] < 2^30, exact in wrapping 32-bit arithmetic
  const int w1 = (int)((unsigned)w[FS_E1 * 32] + (unsigned)rx * (unsigned)w[FS_SX1 * 32] +
                       (unsigned)ry * (unsigned)w[FS_SY1 * 32]);
  const int w2 = (int)((unsigned)w[FS_E2 * 32] + (unsigned)rx * (unsigned)w[FS_SX2 * 32] +
                       (unsigned)ry * (unsigned)w[FS_SY2 * 32]);
  const float k1 = __int_as_float(w[FS_K1 * 32]), k2 = __int_as_float(w[FS_K2 * 32]);
  const int d1 = w[FS_D1 * 32], d2 = w[FS_D2 * 32], sA = w[FS_A * 32];
  int q = __float2int_rd(__fmaf_rn((float)w1, k1, (float)w2 * k2));
  if (sA > 0) {
    int r = (int)((unsigned)w1 * (unsigned)d1 + (unsigned)w2 * (unsigned)d2 - (unsigned)q * (unsigned)sA);
    for (int it = 0; r < 0 && it < DIV_FIX_LIMIT; ++it) { --q; r += sA; }
    for (int it = 0; r >= sA && it < DIV_FIX_LIMIT; ++it) { ++q; r -= sA; }
  } else {
    const long long A = -(long long)sA;
    long long r = (long long)w1 * d1 + (long long)w2 * d2 - (long long)q * A;
    for (int it = 0; r < 0 && it < DIV_FIX_LIMIT; ++it) { --q; r += A; }
    for (int it = 0; r >= A && it < DIV_FIX_LIMIT; ++it) { ++q; r -= A; }
  }
  // the depth field starts at bit 40: q moves the high word by q << 8
  const unsigned hi = (unsigned)w[FS_KHI * 32] + ((unsigned)q << 8);
  const unsigned long long k = ((unsigned long long)hi << 32) | (unsigned)w[FS_KLO * 32];
  if (k < skey[idx]) atomicMin(skey + idx, k);
}

// Called by every lane of the warp: hands out the warp's covered samples of
// small boxes FRAG_CAP at a time.  Returns the warp's fragment count.
__device__ __forceinline__ unsigned fragment_pass(const SmallBox& b, int bshift_x, int* wst, unsigned long long* skey,
                                                  int lane) {
  if (!__any_sync(FULL_MASK, b.mask != 0u)) return 0u;
  int* list = wst + FST_WORDS * 32;
  const int cnt = __popc(b.mask);
  const MultiSpan m = warp_prefix(cnt, lane);
  int pos = m.incl - cnt;
  unsigned mask = b.mask;
  const int first = b.place & 0xFFFF, bw = b.place >> 16;
  // 65536 / bw to within 2 ulp, floored, plus one: within [65536 / bw, 65536 / bw + 2),
  // which makes (j * M) >> 16 = floor(j / bw) for every j < 32
  const unsigned M = __float2uint_rz(__fdividef(65536.0f, (float)bw)) + 1u;
  for (int base = 0; base < m.total; base += FRAG_CAP) {
    while (mask != 0u && pos < base + FRAG_CAP) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1u;
      const int ry = (int)(((unsigned)j * M) >> 16), rx = j - ry * bw;
      list[pos - base] = (first + (ry << bshift_x) + rx) | (rx << 12) | (ry << 17) | (lane << 22);
      ++pos;
    }
    __syncwarp();
    const int n = min(FRAG_CAP, m.total - base);
    for (int k = lane; k < n; k += 32) fragment_key(wst, (unsigned)list[k], skey);
    __syncwarp();
  }
  return (unsigned)m.total;
}

// A warp covers a large triangle's box 32 pixels at a time; the ballot of
// coverage lets the warp skip groups of pixels with nothing inside.  Each
// lane evaluates the three edge functions of its pixel directly from the
// snapped vertices (two 32x32->64 products per edge), so the warp path holds
// no 64-bit edge increments.
__device__ __forceinline__ unsigned raster_warp(const TriSetup& s, unsigned long long tag, int px0, int px1, int py0,
                                                int py1, int x0, int y0, int bshift_x, unsigned long long* skey,
                                                int lane) {
  const float rA = approx_rcp(f32_from_i64(s.A));
  const int bw = px1 - px0 + 1, n = bw * (py1 - py0 + 1);
  const int dy = 32 / bw, dx = 32 - dy * bw;
  int lx = lane % bw, ly = lane / bw;
  const bool mid = s.A < (1LL << 31);  // the same for the whole warp
  // fill-rule bias of each edge: 1 unless the edge is top-left
  const int b0 = 1 - top_left(s.X2 - s.X1, s.Y2 - s.Y1);
  const int b1 = 1 - top_left(s.X0 - s.X2, s.Y0 - s.Y2);
  const int b2 = 1 - top_left(s.X1 - s.X0, s.Y1 - s.Y0);
  unsigned frags = 0;
  for (int base = 0; base < n; base += 32) {
    const int Px = 256 * (px0 + lx) + 128, Py = 256 * (py0 + ly) + 128;
    const long long w0 = (long long)(s.X2 - s.X1) * (Py - s.Y1) - (long long)(s.Y2 - s.Y1) * (Px - s.X1);
    const long long w1 = (long long)(s.X0 - s.X2) * (Py - s.Y2) - (long long)(s.Y0 - s.Y2) * (Px - s.X2);
    const long long w2 = (long long)(s.X1 - s.X0) * (Py - s.Y0) - (long long)(s.Y1 - s.Y0) * (Px - s.X0);
    const bool cov = base + lane < n && ((w0 - b0) | (w1 - b1) | (w2 - b2)) >= 0;
    const unsigned m = __ballot_sync(FULL_MASK, cov);
    if (m != 0u) {
      if (cov) {
        const int idx = ((py0 + ly - y0) << bshift_x) + (px0 + lx - x0);
        if (mid)
          key_min_mid(skey, idx, (int)w1, (int)w2, s, rA, tag);
        else
          key_min_large(skey, idx, w1, w2, s, rA, tag);
      }
      frags += __popc(m);
    }
    lx += dx; ly += dy;
    if (lx >= bw) { lx -= bw; ++ly; }
  }
  return frags;
}

// Row spans for the large boxes: the covered pixel centres of a row are an
// interval (each edge's test is a half-plane, monotone along the row), so
// a lane per row finds its interval's ends exactly by bisection on the
// edge tests, and the warp then walks only the covered samples, 32 at a
// time, instead of the whole box.  Every covered sample gets the same
// depth key as in raster_warp.
//
// Narrows [lo, hi] to the columns of row Py (16.8 centre) where edge
// (ex, ey) through (Xr, Yr) with fill-rule bias b passes (empty: hi < lo).
__device__ __forceinline__ void clip_span(int ex, int ey, int Xr, int Yr, int b, int Py, int& lo, int& hi) {
  if (lo > hi) return;
  const long long wy = (long long)ex * (Py - Yr) - b;
  // the test at column px: wy - ey (256 px + 128 - Xr) >= 0
  auto pass = [&](int px) { return wy - (long long)ey * (256 * px + 128 - Xr) >= 0; };
  if (ey == 0) {
    if (!pass(lo)) hi = lo - 1;
    return;
  }
  if (ey < 0) {  // the test only turns true along the row: its first passing column
    if (pass(lo)) return;
    if (!pass(hi)) { hi = lo - 1; return; }
    int a = lo, c = hi;  // pass(a) false, pass(c) true; at most 6 halvings for 64 columns
    while (c - a > 1) {
      const int m = (a + c) >> 1;
      if (pass(m)) c = m; else a = m;
    }
    lo = c;
  } else {       // the test only turns false along the row: its last passing column
    if (pass(hi)) return;
    if (!pass(lo)) { hi = lo - 1; return; }
    int a = lo, c = hi;  // pass(a) true, pass(c) false
    while (c - a > 1) {
      const int m = (a + c) >> 1;
      if (pass(m)) a = m; else c = m;
    }
    hi = a;
  }
}

__device__ __forceinline__ unsigned raster_warp_spans(const TriSetup& s, unsigned long long tag, int px0, int px1,
                                                      int py0, int py1, int x0, int y0, int bshift_x,
                                                      unsigned long long* skey, int lane) {
  const float rA = approx_rcp(f32_from_i64(s.A));
  const bool mid = s.A < (1LL << 31);  // the same for the whole warp
  const int b0 = 1 - top_left(s.X2 - s.X1, s.Y2 - s.Y1);
  const int b1 = 1 - top_left(s.X0 - s.X2, s.Y0 - s.Y2);
  const int b2 = 1 - top_left(s.X1 - s.X0, s.Y1 - s.Y0);
  unsigned frags = 0;
  for (int r0 = py0; r0 <= py1; r0 += 32) {  // rows in groups of 32, a lane each
    const int py = r0 + lane;
    int lo = px0, hi = py <= py1 ? px1 : px0 - 1;
    const int Py = 256 * py + 128;
    clip_span(s.X2 - s.X1, s.Y2 - s.Y1, s.X1, s.Y1, b0, Py, lo, hi);
    clip_span(s.X0 - s.X2, s.Y0 - s.Y2, s.X2, s.Y2, b1, Py, lo, hi);
    clip_span(s.X1 - s.X0, s.Y1 - s.Y0, s.X0, s.Y0, b2, Py, lo, hi);
    const int cnt = hi >= lo ? hi - lo + 1 : 0;
    const MultiSpan m = warp_prefix(cnt, lane);
    for (int k0 = 0; k0 < m.total; k0 += 32) {
      const int k = k0 + lane;
      const int owner = pair_owner(m.incl, k < m.total ? k : m.total - 1);
      const int olo = __shfl_sync(FULL_MASK, lo, owner);
      const int ofirst = __shfl_sync(FULL_MASK, m.incl - cnt, owner);
      if (k < m.total) {
        const int px = olo + (k - ofirst), qy = r0 + owner;
        const int Px = 256 * px + 128, Qy = 256 * qy + 128;
        const long long w1 = (long long)(s.X0 - s.X2) * (Qy - s.Y2) - (long long)(s.Y0 - s.Y2) * (Px - s.X2);
        const long long w2 = (long long)(s.X1 - s.X0) * (Qy - s.Y0) - (long long)(s.Y1 - s.Y0) * (Px - s.X0);
        const int idx = ((qy - y0) << bshift_x) + (px - x0);
        if (mid)
          key_min_mid(skey, idx, (int)w1, (int)w2, s, rA, tag);
        else
          key_min_large(skey, idx, w1, w2, s, rA, tag);
      }
    }
    frags += (unsigned)m.total;
  }
  return frags;
}

// ---------------------------------------------------------------- shading
__device__ __forceinline__ uint2 pack_half4(float a, float b, float c, float d) {
  const __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
  uint2 r;
  r.x = *reinterpret_cast<const unsigned*>(&lo);
  r.y = *reinterpret_cast<const unsigned*>(&hi);
  return r;
}

__device__ __forceinline__ void write_empty(const TileScene& p, size_t o) {
  if (p.mode == PIKO_SHADE_GBUFFER) {
    p.gnorm_out[o] = make_uint2(0u, 0u);
    p.galb_out[o] = make_uint2(0u, 0u);
  } else if (p.rgba_out) {
    p.rgba_out[o] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Barycentrics of pixel (x, y) from a record: exact edge functions times
// 1/A.  The record stores 1/A negated when A >= 2^31; below that the pixel's
// edge functions (in [0, A], the pixel being covered) are exact in wrapping
// 32-bit arithmetic.
__device__ __forceinline__ void rec_bary(const int* r, int x, int y, float& b0, float& b1, float& b2) {
  const int Px = 256 * x + 128, Py = 256 * y + 128;
  const int X0 = r[0], Y0 = r[1], X1 = r[2], Y1 = r[3], X2 = r[4], Y2 = r[5];
  const float rAs = __int_as_float(r[R_RA]);
  if (rAs > 0.0f) {
    b1 = (float)edge_fn_wrap32(X2, Y2, X0, Y0, Px, Py) * rAs;
    b2 = (float)edge_fn_wrap32(X0, Y0, X1, Y1, Px, Py) * rAs;
  } else {
    // exact edge functions from 32-bit differences (each below 2^24) widened once
    const long long w1 = (long long)(X0 - X2) * (Py - Y2) - (long long)(Y0 - Y2) * (Px - X2);
    const long long w2 = (long long)(X1 - X0) * (Py - Y0) - (long long)(Y1 - Y0) * (Px - X0);
    b1 = f32_from_i64(w1) * -rAs;
    b2 = f32_from_i64(w2) * -rAs;
  }
  b0 = 1.0f - b1 - b2;
}

// PERSP: perspective-correct barycentrics (the record holds the vertices' 1/w)
template <bool PERSP>
__device__ __forceinline__ void shade_from_record(const TileScene& p, const int* r, int x, int y, size_t o) {
  float b0, b1, b2;
  rec_bary(r, x, y, b0, b1, b2);
  const float* a = reinterpret_cast<const float*>(r + R_ATTR);
  if (PERSP) {
    const float* iw = a + rec_attr_count(p.mode, p.color != nullptr);
    perspective_bary(b0, b1, b2, iw[0], iw[1], iw[2]);
  }
  if (p.mode == PIKO_SHADE_GOURAUD) {
    if (p.rgba_out)
      p.rgba_out[o] = make_float4(b0 * a[0] + b1 * a[3] + b2 * a[6], b0 * a[1] + b1 * a[4] + b2 * a[7],
                                  b0 * a[2] + b1 * a[5] + b2 * a[8], 1.0f);
    return;
  }
  if (p.mode == PIKO_SHADE_LAMBERT) {
    float d = b0 * a[0] + b1 * a[1] + b2 * a[2];  // (sum b_i n_i) . L, by linearity
    if (!p.unclamped) d = fmaxf(d, 0.0f);
    float c0 = 0.80f, c1 = 0.75f, c2 = 0.65f;      // material of Listing 1
    if (p.color) {
      c0 = b0 * a[3] + b1 * a[6] + b2 * a[9];
      c1 = b0 * a[4] + b1 * a[7] + b2 * a[10];
      c2 = b0 * a[5] + b1 * a[8] + b2 * a[11];
    }
    if (p.rgba_out) p.rgba_out[o] = make_float4(c0 * d, c1 * d, c2 * d, 1.0f);
    return;
  }
  const float nx = b0 * a[0] + b1 * a[3] + b2 * a[6];
  const float ny = b0 * a[1] + b1 * a[4] + b2 * a[7];
  const float nz = b0 * a[2] + b1 * a[5] + b2 * a[8];
  float c0 = 0.80f, c1 = 0.75f, c2 = 0.65f;
  if (p.color) {
    c0 = b0 * a[9] + b1 * a[12] + b2 * a[15];
    c1 = b0 * a[10] + b1 * a[13] + b2 * a[16];
    c2 = b0 * a[11] + b1 * a[14] + b2 * a[17];
  }
  p.gnorm_out[o] = pack_half4(nx, ny, nz, 0.0f);
  p.galb_out[o] = pack_half4(c0, c1, c2, 1.0f);
}

// Attributes of a winner with barycentrics (b0, b1, b2) over vertices
// (v0, v1, v2), read from global memory, shaded and written at o.
__device__ __forceinline__ void shade_vertices(const TileScene& p, int v0, int v1, int v2, float b0, float b1,
                                               float b2, size_t o) {
  float c0 = 0.80f, c1 = 0.75f, c2 = 0.65f;
  if (p.color) {
    const float* q0 = p.color + 3 * (size_t)v0;
    const float* q1 = p.color + 3 * (size_t)v1;
    const float* q2 = p.color + 3 * (size_t)v2;
    c0 = b0 * __ldg(q0) + b1 * __ldg(q1) + b2 * __ldg(q2);
    c1 = b0 * __ldg(q0 + 1) + b1 * __ldg(q1 + 1) + b2 * __ldg(q2 + 1);
    c2 = b0 * __ldg(q0 + 2) + b1 * __ldg(q1 + 2) + b2 * __ldg(q2 + 2);
  }
  if (p.mode == PIKO_SHADE_GOURAUD) {
    if (p.rgba_out) p.rgba_out[o] = make_float4(c0, c1, c2, 1.0f);
    return;
  }
  const float* n0 = p.normal + 3 * (size_t)v0;
  const float* n1 = p.normal + 3 * (size_t)v1;
  const float* n2 = p.normal + 3 * (size_t)v2;
  const float nx = b0 * __ldg(n0) + b1 * __ldg(n1) + b2 * __ldg(n2);
  const float ny = b0 * __ldg(n0 + 1) + b1 * __ldg(n1 + 1) + b2 * __ldg(n2 + 1);
  const float nz = b0 * __ldg(n0 + 2) + b1 * __ldg(n1 + 2) + b2 * __ldg(n2 + 2);
  if (p.mode == PIKO_SHADE_GBUFFER) {
    p.gnorm_out[o] = pack_half4(nx, ny, nz, 0.0f);
    p.galb_out[o] = pack_half4(c0, c1, c2, 1.0f);
    return;
  }
  float d = nx * __ldg(p.light) + ny * __ldg(p.light + 1) + nz * __ldg(p.light + 2);
  if (!p.unclamped) d = fmaxf(d, 0.0f);
  if (p.rgba_out) p.rgba_out[o] = make_float4(c0 * d, c1 * d, c2 * d, 1.0f);
}

// Fallback for winners without a record: everything re-read from global
// memory.  CLIP (near/far clipping on): a winner whose vertices the vertex
// stage rejected was clipped, and shades with its clip-space ray weights
// (perspective-correct by construction); one kernel instance per setting so
// that the default path carries none of it.
template <bool PERSP, bool CLIP = false>
__device__ __forceinline__ void shade_from_global(const TileScene& p, unsigned t, int x, int y, size_t o) {
  const int v[3] = {__ldg(p.tris + 3 * (size_t)t), __ldg(p.tris + 3 * (size_t)t + 1),
                    __ldg(p.tris + 3 * (size_t)t + 2)};
  TriSetup s;
  if (!setup_triangle(v[0], v[1], v[2], p.vtx, s)) {
    if (!CLIP || !p.pos) {
      write_empty(p, o);
      return;
    }
    float b0, b1, b2;
    clip_ray_weights(p.pos, p.mvp, p.g.W, p.g.H, v, x, y, b0, b1, b2);
    shade_vertices(p, v[0], v[1], v[2], b0, b1, b2, o);
    return;
  }
  const int Px = 256 * x + 128, Py = 256 * y + 128;
  const long long w1 = (long long)(s.X0 - s.X2) * (Py - s.Y2) - (long long)(s.Y0 - s.Y2) * (Px - s.X2);
  const long long w2 = (long long)(s.X1 - s.X0) * (Py - s.Y0) - (long long)(s.Y1 - s.Y0) * (Px - s.X0);
  const float rA = approx_rcp(f32_from_i64(s.A));
  float b1 = f32_from_i64(w1) * rA, b2 = f32_from_i64(w2) * rA, b0 = 1.0f - b1 - b2;
  if (PERSP) perspective_bary(b0, b1, b2, __ldg(p.invw + s.v0), __ldg(p.invw + s.v1), __ldg(p.invw + s.v2));
  shade_vertices(p, s.v0, s.v1, s.v2, b0, b1, b2, o);
}

// Fills the shared-memory record of one bin entry (PERSP: with 1/w).
template <bool PERSP>
__device__ __forceinline__ void fill_record(const TileScene& p, const TriSetup& s, int* r) {
  r[0] = s.X0; r[1] = s.Y0; r[2] = s.X1; r[3] = s.Y1; r[4] = s.X2; r[5] = s.Y2;
  // 1/A, negated when A >= 2^31 (rec_bary then takes the 64-bit form)
  const float rA = approx_rcp(f32_from_i64(s.A));
  r[R_RA] = __float_as_int(s.A < (1LL << 31) ? rA : -rA);
  float* a = reinterpret_cast<float*>(r + R_ATTR);
  const int v[3] = {s.v0, s.v1, s.v2};
  if (PERSP) {
    float* iw = a + rec_attr_count(p.mode, p.color != nullptr);
#pragma unroll
    for (int j = 0; j < 3; ++j) iw[j] = __ldg(p.invw + v[j]);
  }
  if (p.mode == PIKO_SHADE_LAMBERT) {
#pragma unroll
    for (int j = 0; j < 3; ++j) a[j] = __ldg(p.vdot + v[j]);
    if (p.color) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float* c = p.color + 3 * (size_t)v[j];
        a[3 + 3 * j] = __ldg(c); a[4 + 3 * j] = __ldg(c + 1); a[5 + 3 * j] = __ldg(c + 2);
      }
    }
    return;
  }
  const int coff = p.mode == PIKO_SHADE_GOURAUD ? 0 : 9;
  if (p.mode == PIKO_SHADE_GBUFFER) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float* n = p.normal + 3 * (size_t)v[j];
      a[3 * j] = __ldg(n); a[3 * j + 1] = __ldg(n + 1); a[3 * j + 2] = __ldg(n + 2);
    }
  }
  if (p.color) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float* c = p.color + 3 * (size_t)v[j];
      a[coff + 3 * j] = __ldg(c); a[coff + 3 * j + 1] = __ldg(c + 1); a[coff + 3 * j + 2] = __ldg(c + 2);
    }
  }
}

// t is the scene-local triangle index
__device__ __forceinline__ void load_setup(const TileScene& p, unsigned t, TriSetup& s) {
  setup_triangle(__ldg(p.tris + 3 * (size_t)t), __ldg(p.tris + 3 * (size_t)t + 1), __ldg(p.tris + 3 * (size_t)t + 2),
                 p.vtx, s);
}


// Process one tile: tile is the scene-local tile index, [beg, end) its range
// in bin_tris.  Called by every thread of the CTA (nt threads, a power of
// two); contains CTA barriers.  big_base tracks the large-triangle ring.
// PERSP: perspective-correct attributes (p.invw set); CLIP: near/far
// clipping (entries T.. are clipped sub-triangles); one kernel instance per
// setting so that the default path carries none of either.
template <bool STATS, bool PERSP = false, bool CLIP = false>
__device__ __forceinline__ void process_tile(const TileScene& p, int tile, unsigned beg, unsigned end,
                                             const unsigned* __restrict__ bin_tris, const TileSmem& sm,
                                             unsigned& big_base, TileStats& st) {
  const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const int bin_w = 1 << p.g.bshift_x, bin_h = 1 << p.g.bshift_y;
  const int bin_px = bin_w * bin_h;
  const unsigned no_slot = (1u << p.slot_bits) - 1u;
  const int tx = tile % p.g.nbx, ty = tile / p.g.nbx;
  const int x0 = tx << p.g.bshift_x, y0 = ty << p.g.bshift_y;
  const int x1 = min(x0 + bin_w, p.g.W) - 1, y1 = min(y0 + bin_h, p.g.H) - 1;
  unsigned long long* skey = sm.skey;
  int* wst = sm.sfrag + warp * FRAG_WARP_WORDS;
  for (unsigned c = beg; c < end; c += nt) {
    const unsigned i = c + tid;
    bool pushed = false;
    SmallBox sb;
    sb.mask = 0u;
    if (i < end) {
      unsigned t = __ldg(bin_tris + i) - (unsigned)p.tri_base;
      unsigned slot = (i - beg) < (unsigned)p.nslots ? (i - beg) : no_slot;
      TriSetup s;
      if (CLIP && t >= (unsigned)p.T) {
        // a clipped sub-triangle: its points, the key of its triangle, no
        // record (the winner shades from its triangle's clip coordinates)
        const int4* c = p.clip_tris + 3 * (size_t)(t - (unsigned)p.T);
        setup_points(__ldg(c), __ldg(c + 1), __ldg(c + 2), s);
        t = __ldg(p.clip_orig + (t - (unsigned)p.T));
        slot = no_slot;
      } else {
        load_setup(p, t, s);
      }
      if (slot != no_slot) fill_record<PERSP>(p, s, sm.srec + slot * p.rec_stride);
      const int minX = min(s.X0, min(s.X1, s.X2)), maxX = max(s.X0, max(s.X1, s.X2));
      const int minY = min(s.Y0, min(s.Y1, s.Y2)), maxY = max(s.Y0, max(s.Y1, s.Y2));
      int px0, px1, py0, py1;
      centre_range(minX, maxX, x0, x1, px0, px1);
      centre_range(minY, maxY, y0, y1, py0, py1);
      if (px0 <= px1 && py0 <= py1) {
        const int npx = (px1 - px0 + 1) * (py1 - py0 + 1);
        const unsigned long long tag = ((unsigned long long)t << p.slot_bits) | slot;
        if (STATS) st.tests += npx;
        if (npx <= p.small_px) {
          unsigned f = 0u;
          if (maxX - minX < 32768 && maxY - minY < 32768) {
            if (npx <= 32)  // coverage only; the warp's fragment_pass takes the depths
              small_box(s, tag, px0, px1, py0, py1, x0, y0, p.g.bshift_x, wst, lane, sb);
            else
              f = raster_thread32(s, tag, px0, px1, py0, py1, x0, y0, p.g.bshift_x, skey);
          } else {
            f = raster_thread64(s, tag, px0, px1, py0, py1, x0, y0, p.g.bshift_x, skey);
          }
          if (STATS) st.frags += f;
        } else {
          // the ring counter only ever grows; with nt a power of two the ring
          // index stays consistent across its 2^32 wrap
          const unsigned q = atomicAdd(sm.s_nbig, 1u);
          sm.sbig[q & (nt - 1)] = tid;
          int* e = wst + lane;
          e[BG_X0 * 32] = s.X0; e[BG_Y0 * 32] = s.Y0; e[BG_X1 * 32] = s.X1; e[BG_Y1 * 32] = s.Y1;
          e[BG_X2 * 32] = s.X2; e[BG_Y2 * 32] = s.Y2;
          e[BG_Z0 * 32] = s.Z0; e[BG_Z1 * 32] = s.Z1; e[BG_Z2 * 32] = s.Z2;
          e[BG_ALO * 32] = (int)(unsigned)(s.A & 0xFFFFFFFFll); e[BG_AHI * 32] = (int)(s.A >> 32);
          e[BG_T * 32] = (int)t; e[BG_SLOT * 32] = (int)slot;
          pushed = true;
        }
      }
    }
    {
      const unsigned f = fragment_pass(sb, p.g.bshift_x, wst, skey, lane);
      if (STATS && lane == 0) st.frags += f;
    }
    // every thread gets the same count of queued large triangles
    const unsigned nbig = (unsigned)__syncthreads_count(pushed);
    if (nbig != 0u) {
      for (unsigned q = warp; q < nbig; q += nwarps) {
        const int owner = sm.sbig[(big_base + q) & (nt - 1)];
        const int* e = sm.sfrag + (owner >> 5) * FRAG_WARP_WORDS + (owner & 31);
        TriSetup s;
        s.X0 = e[BG_X0 * 32]; s.Y0 = e[BG_Y0 * 32]; s.X1 = e[BG_X1 * 32]; s.Y1 = e[BG_Y1 * 32];
        s.X2 = e[BG_X2 * 32]; s.Y2 = e[BG_Y2 * 32];
        s.Z0 = e[BG_Z0 * 32]; s.Z1 = e[BG_Z1 * 32]; s.Z2 = e[BG_Z2 * 32];
        s.A = (long long)(((unsigned long long)(unsigned)e[BG_AHI * 32] << 32) | (unsigned)e[BG_ALO * 32]);
        s.v0 = s.v1 = s.v2 = 0;  // not needed to rasterize
        const unsigned t = (unsigned)e[BG_T * 32], slot = (unsigned)e[BG_SLOT * 32];
        int px0, px1, py0, py1;
        centre_range(min(s.X0, min(s.X1, s.X2)), max(s.X0, max(s.X1, s.X2)), x0, x1, px0, px1);
        centre_range(min(s.Y0, min(s.Y1, s.Y2)), max(s.Y0, max(s.Y1, s.Y2)), y0, y1, py0, py1);
        const unsigned long long tag = ((unsigned long long)t << p.slot_bits) | slot;
        const unsigned f = (px1 - px0 + 1) * (py1 - py0 + 1) >= PIKO_SPAN_MIN_PX
                               ? raster_warp_spans(s, tag, px0, px1, py0, py1, x0, y0, p.g.bshift_x, skey, lane)
                               : raster_warp(s, tag, px0, px1, py0, py1, x0, y0, p.g.bshift_x, skey, lane);
        if (STATS && lane == 0) st.frags += f;
      }
      big_base += nbig;
      __syncthreads();
    }
  }
  // shade, write, and leave the key tile cleared for the next tile
  for (int i = tid; i < bin_px; i += nt) {
    const unsigned long long k = skey[i];
    skey[i] = KEY_EMPTY;
    const int x = x0 + (i & (bin_w - 1)), y = y0 + (i >> p.g.bshift_x);
    if (x > x1 || y > y1) continue;
    const size_t o = (size_t)y * p.g.W + x;
    if (k == KEY_EMPTY) {
      p.key_out[o] = KEY_EMPTY;
      write_empty(p, o);
      continue;
    }
    const unsigned z = (unsigned)(k >> 40);
    // the triangle field sits between the slot and the depth: 40 - slot_bits wide
    const unsigned t = (unsigned)((k >> p.slot_bits) & ((1ull << (40 - p.slot_bits)) - 1ull));
    const unsigned slot = (unsigned)(k & no_slot);
    p.key_out[o] = ((unsigned long long)z << 32) | t;
    if (STATS) ++st.shaded;
    if (slot != no_slot)
      shade_from_record<PERSP>(p, sm.srec + slot * p.rec_stride, x, y, o);
    else
      shade_from_global<PERSP, CLIP>(p, t, x, y, o);
  }
  __syncthreads();
}

// Record layout of a scene: slot bits below the triangle index (2^id_bits > T,
// so no key equals the all-ones empty key), records per tile and words per
// record (odd, so that distinct records fall in distinct banks).  want_slots
// (0: as many as allowed) sizes the record area: shared memory taken by
// records is taken from L1, which serves the kernel's gathers, so records
// are sized for the tiles' typical entry count rather than the largest.
// persp adds the three vertices' 1/w (perspective-correct attributes).
inline void tile_layout(int num_triangles, int bin_px, int mode, bool has_color, bool persp, int max_slots,
                        int& slot_bits, int& nslots, int& rec_stride, int want_slots = 0) {
  int id_bits = 1;
  while (id_bits < 32 && (1LL << id_bits) <= (long long)num_triangles) ++id_bits;
  slot_bits = 40 - id_bits < 16 ? 40 - id_bits : 16;
  int want = bin_px <= 256 ? 255 : max_slots;
  if (want_slots > 0 && want_slots < want) want = want_slots;
  const int cap = (1 << slot_bits) - 1;
  nslots = want < cap ? want : cap;
  rec_stride = R_ATTR + rec_attr_count(mode, has_color) + (persp ? 3 : 0);
  if ((rec_stride & 1) == 0) ++rec_stride;
}

inline size_t tile_smem_bytes(int bin_px, int threads, int nslots, int rec_stride) {
  return (size_t)bin_px * 8 + (size_t)threads * 4 + (size_t)(threads / 32) * FRAG_WARP_WORDS * 4 +
         (size_t)nslots * rec_stride * 4;
}

}  // namespace piko
