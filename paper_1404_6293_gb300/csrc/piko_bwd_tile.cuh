// piko_bwd_tile.cuh -- gradients of the shading, accumulated per screen tile;
// shared by the single-scene and the batch backward kernels.
//
// Visibility is held fixed by the forward key buffer, so coverage stays exact
// integer arithmetic and only the fragment shader is differentiated: for the
// Lambert shader of Listing 1 (rgb = albedo * s, s = max(0, n . L),
// n = sum b_i n_i, albedo = sum b_i c_i) and for Gouraud (rgb = sum b_i c_i).
// Per pixel, with g = dLoss/drgb:
//   dL/dc_i += s * b_i * g        (Gouraud: b_i * g)
//   dL/dn_i += (g . albedo) b_i L   when s > 0 (or unclamped)
//   dL/dL   += (g . albedo) n
//
// A warp takes a 16 x 16 or 16 x 32 tile (backward_warp_tile, below) with no
// CTA barrier: the warps of a CTA work on separate tiles.  Each lane walks a
// column of the tile and keeps, for as long as its pixels keep the same
// winning triangle (a run), that triangle's setup (vertex indices, snapped
// positions, 2 x area) and the sums of its 12 per-pixel terms (below) in
// registers; a run that ends is summed with the other lanes' runs of the same
// triangle and added to the gradient arrays with one set of atomics.  A
// triangle is set up once per run rather than per pixel, and a triangle that
// covers a column of the tile is flushed once for it.
#pragma once

#include "piko_internal.cuh"

namespace piko {

// Rows per tile: the batch backward takes 16 x 32 tiles, longer column runs
// per lane (256-scene batch 5.03 -> 4.87 ms, sphere views 0.672 -> 0.663 ms;
// 16 x 64: 4.95 and 0.79 ms); a single scene keeps 16 x 16, twice the tiles
// for its one frame (with 16 x 32 the 256-scene per-scene loop took 31.2 ms
// against 26.3).
#ifndef PIKO_BWD_TILE_H
#define PIKO_BWD_TILE_H 16
#endif
#ifndef PIKO_BATCH_BWD_TILE_H
#define PIKO_BATCH_BWD_TILE_H 32
#endif
constexpr int BWD_TILE_W = 16;                           // pixels per tile row (a warp pass covers two rows)
constexpr int BWD_TILE_H = PIKO_BWD_TILE_H;              // rows per tile, single scene
constexpr int BATCH_BWD_TILE_H = PIKO_BATCH_BWD_TILE_H;  // rows per tile, batch
constexpr int BWD_THREADS = 256;             // CTA size of the backward kernels (8 warps, a tile each)
// Terms per pixel: q = 3 j + c (c < 3) is g_c s b_j, the colour gradient of
// vertex j (g_c b_j for Gouraud); q = 9 + j is G b_j with G = g . albedo
// (0 where the clamp is inactive).  The normal and light gradients are
// linear in the G b_j sums: dL/dn_j = L sum(G b_j) and dL/dL = sum_j n_j
// sum(G b_j), so they are formed once per slot from the sums.
constexpr int BWD_VALS = 12;
constexpr unsigned BWD_NONE = 0xFFFFFFFFu;

struct BwdScene {
  int W, H, mode, unclamped, T, V;
  const int* tris;
  const int4* vtx;
  const float* color;
  const float* normal;
  const float* light;
  const float* invw;  // 1 / clip w per vertex: perspective-correct attributes (NULL: screen-space)
  const float4* pos;  // near/far clipping: positions and matrix of clipped winners (NULL: off)
  const float* mvp;
  const unsigned long long* key;
  const float4* dl;
  float* dcolor;
  float* dnormal;
  float* dlight;
};

// ---------------------------------------------------------------- warp form
// One warp takes a BWD_TILE_W x TILE_H tile in passes of 16 x 2 pixels:
// lane l follows column l mod 16 down the rows of parity l / 16.  A run that
// ends is flushed (bwd_run_flush): lanes ending runs of the same triangle
// are summed through the warp's staging area, one lane per term, with one
// set of atomics per group, and runs of one or two lanes add their own terms.

// The setup of a lane's current triangle: oriented snapped positions, A
// (lo, hi words), 1/A, vertex ids, n_j . L (Lambert) and kind (0: nothing to
// add, 1: covered by its snapped edges, 2: clipped winner, ray weights).
struct BwdRun {
  int X0, Y0, X1, Y1, X2, Y2, alo, ahi;
  float rA, d0, d1, d2;
  int v0, v1, v2, kind;
};

__device__ __forceinline__ BwdRun bwd_run_shfl(const BwdRun& r, int src) {
  BwdRun o;
  o.X0 = __shfl_sync(FULL_MASK, r.X0, src); o.Y0 = __shfl_sync(FULL_MASK, r.Y0, src);
  o.X1 = __shfl_sync(FULL_MASK, r.X1, src); o.Y1 = __shfl_sync(FULL_MASK, r.Y1, src);
  o.X2 = __shfl_sync(FULL_MASK, r.X2, src); o.Y2 = __shfl_sync(FULL_MASK, r.Y2, src);
  o.alo = __shfl_sync(FULL_MASK, r.alo, src); o.ahi = __shfl_sync(FULL_MASK, r.ahi, src);
  o.rA = __shfl_sync(FULL_MASK, r.rA, src);
  o.d0 = __shfl_sync(FULL_MASK, r.d0, src); o.d1 = __shfl_sync(FULL_MASK, r.d1, src);
  o.d2 = __shfl_sync(FULL_MASK, r.d2, src);
  o.v0 = __shfl_sync(FULL_MASK, r.v0, src); o.v1 = __shfl_sync(FULL_MASK, r.v1, src);
  o.v2 = __shfl_sync(FULL_MASK, r.v2, src);
  o.kind = __shfl_sync(FULL_MASK, r.kind, src);
  return o;
}

// Sets up triangle t (a winner of this scene) for the backward pass.  CLIP:
// near/far clipping may be on (sc.pos set).
template <bool CLIP>
__device__ __forceinline__ void bwd_run_setup(const BwdScene& sc, unsigned t, float L0, float L1, float L2,
                                              BwdRun& r) {
  const int ia = __ldg(sc.tris + 3 * (size_t)t), ib = __ldg(sc.tris + 3 * (size_t)t + 1),
            ic = __ldg(sc.tris + 3 * (size_t)t + 2);
  const bool in_range = ia >= 0 && ia < sc.V && ib >= 0 && ib < sc.V && ic >= 0 && ic < sc.V;
  TriSetup ts;
  const bool ok = in_range && setup_triangle(ia, ib, ic, sc.vtx, ts);
  // a winner the vertex stage rejected was clipped: per-pixel ray weights
  const bool clipped = CLIP && !ok && in_range && sc.pos;
  r.kind = ok ? 1 : (clipped ? 2 : 0);
  if (ok) {
    r.X0 = ts.X0; r.Y0 = ts.Y0; r.X1 = ts.X1; r.Y1 = ts.Y1; r.X2 = ts.X2; r.Y2 = ts.Y2;
    r.v0 = ts.v0; r.v1 = ts.v1; r.v2 = ts.v2;
    r.alo = (int)(unsigned)(ts.A & 0xFFFFFFFFll);
    r.ahi = (int)(ts.A >> 32);
    r.rA = __frcp_rn(f32_from_i64(ts.A));
  } else {
    r.v0 = ia; r.v1 = ib; r.v2 = ic;
  }
  if (r.kind != 0 && sc.mode == PIKO_SHADE_LAMBERT) {
    const float* n0 = sc.normal + 3 * (size_t)r.v0;
    const float* n1 = sc.normal + 3 * (size_t)r.v1;
    const float* n2 = sc.normal + 3 * (size_t)r.v2;
    r.d0 = __ldg(n0) * L0 + __ldg(n0 + 1) * L1 + __ldg(n0 + 2) * L2;
    r.d1 = __ldg(n1) * L0 + __ldg(n1 + 1) * L1 + __ldg(n1 + 2) * L2;
    r.d2 = __ldg(n2) * L0 + __ldg(n2 + 1) * L1 + __ldg(n2 + 2) * L2;
  }
}

// Adds the 12 terms of pixel (x, y), covered by run r, with dL/drgba g, to acc.
template <bool PERSP, bool CLIP>
__device__ __forceinline__ void bwd_run_terms(const BwdScene& sc, const BwdRun& r, int x, int y, const float4 g,
                                              float (&acc)[BWD_VALS]) {
  const int vid[3] = {r.v0, r.v1, r.v2};
  float b[3];
  if (CLIP && r.kind == 2) {
    clip_ray_weights(sc.pos, sc.mvp, sc.W, sc.H, vid, x, y, b[0], b[1], b[2]);
  } else if (r.ahi == 0 && r.alo >= 0) {
    // A < 2^31: the covered pixel's edge functions lie in [0, A], exact in
    // wrapping 32-bit arithmetic
    const int Px = 256 * x + 128, Py = 256 * y + 128;
    const int w1 = edge_fn_wrap32(r.X2, r.Y2, r.X0, r.Y0, Px, Py), w2 = edge_fn_wrap32(r.X0, r.Y0, r.X1, r.Y1, Px, Py);
    const int w0 = r.alo - w1 - w2;  // the three edge functions sum to A
    b[0] = (float)w0 * r.rA; b[1] = (float)w1 * r.rA; b[2] = (float)w2 * r.rA;
  } else {
    const long long A = (long long)(((unsigned long long)(unsigned)r.ahi << 32) | (unsigned)r.alo);
    const long long Px = 256LL * x + 128, Py = 256LL * y + 128;
    const long long w1 = (long long)(r.X0 - r.X2) * (Py - r.Y2) - (long long)(r.Y0 - r.Y2) * (Px - r.X2);
    const long long w2 = (long long)(r.X1 - r.X0) * (Py - r.Y0) - (long long)(r.Y1 - r.Y0) * (Px - r.X0);
    const long long w0 = A - w1 - w2;
    b[0] = f32_from_i64(w0) * r.rA; b[1] = f32_from_i64(w1) * r.rA; b[2] = f32_from_i64(w2) * r.rA;
  }
  if (PERSP && r.kind == 1)
    perspective_bary(b[0], b[1], b[2], __ldg(sc.invw + vid[0]), __ldg(sc.invw + vid[1]), __ldg(sc.invw + vid[2]));
  if (sc.mode == PIKO_SHADE_GOURAUD) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      acc[3 * j] += g.x * b[j]; acc[3 * j + 1] += g.y * b[j]; acc[3 * j + 2] += g.z * b[j];
    }
    return;
  }
  float a0 = 0.80f, a1 = 0.75f, a2 = 0.65f;  // material of Listing 1 without colours
  if (sc.color) {
    a0 = a1 = a2 = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float* c = sc.color + 3 * (size_t)vid[j];
      a0 += b[j] * __ldg(c); a1 += b[j] * __ldg(c + 1); a2 += b[j] * __ldg(c + 2);
    }
  }
  // n . L = sum_j b_j (n_j . L), by linearity
  const float d = b[0] * r.d0 + b[1] * r.d1 + b[2] * r.d2;
  const bool active = sc.unclamped || d > 0.f;
  const float sh = sc.unclamped ? d : fmaxf(d, 0.f);
  const float G = active ? (g.x * a0 + g.y * a1 + g.z * a2) : 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    if (sc.color) {
      acc[3 * j] += g.x * sh * b[j]; acc[3 * j + 1] += g.y * sh * b[j]; acc[3 * j + 2] += g.z * sh * b[j];
    }
    acc[9 + j] += G * b[j];
  }
}

// Adds term q (see BWD_VALS) with value val of a triangle whose vertex j (the
// vertex of term q) is vj to the scene's gradients: a colour term goes to
// dL/dc of the vertex; a G b_j sum goes to dL/dn_j (times L) and, when
// `light` is set, to this thread's share of dL/dL (times n_j).
__device__ __forceinline__ void bwd_add_term_v(const BwdScene& sc, int vj, int q, float val, bool has_c, bool has_n,
                                               bool light, float L0, float L1, float L2, float& gl0, float& gl1,
                                               float& gl2) {
  if (q < 9) {
    if (has_c) atomicAdd(sc.dcolor + 3 * (size_t)vj + (q % 3), val);
    return;
  }
  const size_t vb = 3 * (size_t)vj;
  if (has_n) {
    atomicAdd(sc.dnormal + vb, val * L0);
    atomicAdd(sc.dnormal + vb + 1, val * L1);
    atomicAdd(sc.dnormal + vb + 2, val * L2);
  }
  if (light) {
    gl0 += val * __ldg(sc.normal + vb);
    gl1 += val * __ldg(sc.normal + vb + 1);
    gl2 += val * __ldg(sc.normal + vb + 2);
  }
}

// Flushes the runs of the lanes with fl set (t: their triangle, r: its
// setup, acc: their sums, cleared here).  Warp-collective.
__device__ __forceinline__ void bwd_run_flush(const BwdScene& sc, bool fl, unsigned t, const BwdRun& r,
                                              float (&acc)[BWD_VALS], float (*stage)[33], bool has_c, bool has_n,
                                              bool has_l, float L0, float L1, float L2, float& gl0, float& gl1,
                                              float& gl2) {
  const int lane = threadIdx.x & 31;
  const unsigned grp = __match_any_sync(FULL_MASK, fl ? t : BWD_NONE);
  const bool own = fl && __popc(grp) <= 2;
  if (own) {
    const int vid[3] = {r.v0, r.v1, r.v2};
#pragma unroll
    for (int q = 0; q < BWD_VALS; ++q)
      if (acc[q] != 0.f)
        bwd_add_term_v(sc, vid[q < 9 ? q / 3 : q - 9], q, acc[q], has_c, has_n, has_l, L0, L1, L2, gl0, gl1, gl2);
  }
  unsigned big = __ballot_sync(FULL_MASK, fl && !own);
  if (big != 0u) {
#pragma unroll
    for (int q = 0; q < BWD_VALS; ++q) stage[q][lane] = acc[q];
    __syncwarp();
    // every round removes at least the round's leader lane
    for (int round = 0; big != 0u && round < 32; ++round) {
      const int ld = __ffs(big) - 1;
      const unsigned gm = __shfl_sync(FULL_MASK, grp, ld);
      const int u0 = __shfl_sync(FULL_MASK, r.v0, ld), u1 = __shfl_sync(FULL_MASK, r.v1, ld),
                u2 = __shfl_sync(FULL_MASK, r.v2, ld);
      big &= ~gm;
      if (lane < BWD_VALS) {
        float sum = 0.f;
        for (unsigned m = gm; m; m &= m - 1) sum += stage[lane][__ffs(m) - 1];
        const int j = lane < 9 ? lane / 3 : lane - 9;
        if (sum != 0.f)
          bwd_add_term_v(sc, j == 0 ? u0 : (j == 1 ? u1 : u2), lane, sum, has_c, has_n, has_l, L0, L1, L2, gl0, gl1,
                         gl2);
      }
    }
    __syncwarp();  // the staging area is rewritten by the next flush
  }
  if (fl) {
#pragma unroll
    for (int q = 0; q < BWD_VALS; ++q) acc[q] = 0.f;
  }
}

// One tile with its top-left pixel (x0, y0), taken by one warp (all 32 lanes
// call it with the same arguments); stage is the warp's own staging area.
// The tile's share of dL/dL is added at its end.  A triangle that starts a
// run is set up by the lowest lane of the warp that holds it and broadcast to
// the lanes that need it; a lane whose run goes on keeps its setup.
// CLIP: near/far clipping may be on (sc.pos set).
template <bool PERSP = false, bool CLIP = false, int TILE_H = BWD_TILE_H>
__device__ __forceinline__ void backward_warp_tile(const BwdScene& sc, int x0, int y0, float (*stage)[33], float L0,
                                                   float L1, float L2) {
  const int lane = threadIdx.x & 31;
  const bool has_c = sc.dcolor != nullptr && (sc.mode == PIKO_SHADE_GOURAUD || sc.color != nullptr);
  const bool has_n = sc.dnormal != nullptr && sc.mode == PIKO_SHADE_LAMBERT;
  const bool has_l = sc.dlight != nullptr && sc.mode == PIKO_SHADE_LAMBERT;
  float gl0 = 0.f, gl1 = 0.f, gl2 = 0.f;
  float acc[BWD_VALS];
#pragma unroll
  for (int q = 0; q < BWD_VALS; ++q) acc[q] = 0.f;
  BwdRun r = {0, 0, 0, 0, 0, 0, 0, 0, 0.f, 0.f, 0.f, 0.f, 0, 0, 0, 0};
  unsigned cur = BWD_NONE;
  const int x = x0 + (lane & 15);
  // the triangle word (low half) of the next pass's key is loaded a pass
  // ahead; an empty key's word is all ones
  const unsigned* kw = reinterpret_cast<const unsigned*>(sc.key);
  unsigned knext = x < sc.W && y0 + (lane >> 4) < sc.H ? __ldg(kw + 2 * ((size_t)(y0 + (lane >> 4)) * sc.W + x))
                                                       : BWD_NONE;
  for (int pass = 0; pass < TILE_H / 2; ++pass) {
    const int y = y0 + 2 * pass + (lane >> 4);
    const size_t o = (size_t)y * sc.W + x;
    // a key naming a triangle outside this scene contributes nothing (it
    // cannot come from this scene's forward)
    const unsigned t = knext < (unsigned)sc.T ? knext : BWD_NONE;
    if (pass + 1 < TILE_H / 2)
      knext = x < sc.W && y + 2 < sc.H ? __ldg(kw + 2 * (o + 2 * (size_t)sc.W)) : BWD_NONE;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
    if (t != BWD_NONE) g = __ldg(sc.dl + o);  // issued before the flush and setup it does not need
    const bool change = t != cur;
    const bool ends = change && r.kind != 0;
    if (__any_sync(FULL_MASK, ends))
      bwd_run_flush(sc, ends, cur, r, acc, stage, has_c, has_n, has_l, L0, L1, L2, gl0, gl1, gl2);
    const bool need = change && t != BWD_NONE;
    if (__any_sync(FULL_MASK, need)) {
      const int leader = __ffs(__match_any_sync(FULL_MASK, t)) - 1;
      // a leader whose run goes on already holds the setup
      if (need && lane == leader) bwd_run_setup<CLIP>(sc, t, L0, L1, L2, r);
      const BwdRun s = bwd_run_shfl(r, leader);
      if (need) r = s;
    }
    cur = t;
    if (t == BWD_NONE) r.kind = 0;
    if (r.kind != 0) bwd_run_terms<PERSP, CLIP>(sc, r, x, y, g, acc);
  }
  const bool ends = r.kind != 0;
  if (__any_sync(FULL_MASK, ends))
    bwd_run_flush(sc, ends, cur, r, acc, stage, has_c, has_n, has_l, L0, L1, L2, gl0, gl1, gl2);
  if (has_l) {
    for (int o = 16; o > 0; o >>= 1) {
      gl0 += __shfl_xor_sync(FULL_MASK, gl0, o);
      gl1 += __shfl_xor_sync(FULL_MASK, gl1, o);
      gl2 += __shfl_xor_sync(FULL_MASK, gl2, o);
    }
    if (lane == 0) {
      if (gl0 != 0.f) atomicAdd(sc.dlight, gl0);
      if (gl1 != 0.f) atomicAdd(sc.dlight + 1, gl1);
      if (gl2 != 0.f) atomicAdd(sc.dlight + 2, gl2);
    }
  }
}

}  // namespace piko
