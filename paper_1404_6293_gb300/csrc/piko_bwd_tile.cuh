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
// One CTA of BWD_THREADS threads takes a 16-pixel-wide tile, one pixel per thread:
//  1. the distinct winning triangles of the tile go into a shared hash table
//     (one insert per group of lanes with the same triangle);
//  2. the table is compacted into slots and each slot's triangle is set up
//     once (vertex indices, snapped positions, 2 x area);
//  3. every pixel computes its 12 terms (below) from its slot's setup; the
//     lanes of a warp that share a slot are summed, one lane per term, into
//     the slot's shared accumulators;
//  4. each slot then issues its gradient atomics (9 colour, 9 normal) and
//     adds its share of the light gradient.
// So the setup runs once per (tile, visible triangle) and the global atomics
// number 18 per (tile, visible triangle) instead of per pixel group.  Tiles of
// tiny triangles (more than BWD_DIRECT_SLOTS of them) add their terms to the
// gradients directly, per pixel or per group of lanes.
#pragma once

#include "piko_internal.cuh"

namespace piko {

#ifndef PIKO_BWD_TILE_H
#define PIKO_BWD_TILE_H 16
#endif
constexpr int BWD_TILE_W = 16;               // pixels per tile row (a warp covers two rows)
constexpr int BWD_TILE_H = PIKO_BWD_TILE_H;  // rows per tile
constexpr int BWD_THREADS = BWD_TILE_W * BWD_TILE_H;
constexpr int BWD_HASH_BITS = BWD_THREADS > 128 ? 9 : 8;
constexpr int BWD_HASH = 1 << BWD_HASH_BITS;  // twice the most distinct triangles a tile can hold
// Terms per pixel: q = 3 j + c (c < 3) is g_c s b_j, the colour gradient of
// vertex j (g_c b_j for Gouraud); q = 9 + j is G b_j with G = g . albedo
// (0 where the clamp is inactive).  The normal and light gradients are
// linear in the G b_j sums: dL/dn_j = L sum(G b_j) and dL/dL = sum_j n_j
// sum(G b_j), so they are formed once per slot from the sums.
constexpr int BWD_VALS = 12;
constexpr unsigned BWD_NONE = 0xFFFFFFFFu;

// per-slot words: oriented X0 Y0 X1 Y1 X2 Y2, vertex ids v0 v1 v2, A (lo, hi),
// the triangle id (replaced by 1/A once the slot is set up), a valid flag and
// n_j . L of the three vertices (Lambert); 17 words (odd: distinct slots fall
// in distinct banks)
constexpr int RB_V = 6, RB_ALO = 9, RB_AHI = 10, RB_T = 11, RB_OK = 12, RB_VD = 13, BWD_REC = 17;

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

// Tiles with more distinct triangles than this (under 3 pixels per triangle)
// skip the shared accumulators: their slots would each collect only a pixel
// or two, so the terms go straight to the gradient arrays.
constexpr int BWD_DIRECT_SLOTS = 96;

struct BwdSmem {
  unsigned hkey[BWD_HASH];
  unsigned short hslot[BWD_HASH];
  int rec[BWD_THREADS * BWD_REC];
  float acc[BWD_DIRECT_SLOTS * BWD_VALS];  // only tiles with at most BWD_DIRECT_SLOTS slots accumulate here
  float stage[BWD_THREADS / 32][BWD_VALS][33];  // padded: lane q reads row q, column m
  float lred[BWD_THREADS / 32][3];
  int nslot;
};

__device__ __forceinline__ void bwd_clear(BwdSmem& sm) {
  for (int e = threadIdx.x; e < BWD_HASH; e += blockDim.x) sm.hkey[e] = BWD_NONE;
  if (threadIdx.x == 0) sm.nslot = 0;
}

// Sums the CTA's light-gradient shares (all threads call it; it has barriers).
__device__ __forceinline__ void bwd_flush_light(BwdSmem& sm, float* dlight, float& gl0, float& gl1, float& gl2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    gl0 += __shfl_xor_sync(FULL_MASK, gl0, o);
    gl1 += __shfl_xor_sync(FULL_MASK, gl1, o);
    gl2 += __shfl_xor_sync(FULL_MASK, gl2, o);
  }
  if (lane == 0) {
    sm.lred[warp][0] = gl0; sm.lred[warp][1] = gl1; sm.lred[warp][2] = gl2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float a = 0.f;
    for (int w = 0; w < BWD_THREADS / 32; ++w) a += sm.lred[w][threadIdx.x];
    if (a != 0.f) atomicAdd(dlight + threadIdx.x, a);
  }
  gl0 = gl1 = gl2 = 0.f;
  __syncthreads();
}

// Adds term q of slot record r to the scene's gradients: a colour term goes
// to dL/dc of its vertex; a G b_j sum goes to dL/dn_j (times L) and, when
// `light` is set, to this thread's share of dL/dL (times n_j).
__device__ __forceinline__ void bwd_add_term(const BwdScene& sc, const int* r, int q, float val, bool has_c,
                                             bool has_n, bool light, float L0, float L1, float L2, float& gl0,
                                             float& gl1, float& gl2) {
  if (q < 9) {
    const int j = q / 3, c = q - 3 * j;
    if (has_c) atomicAdd(sc.dcolor + 3 * (size_t)r[RB_V + j] + c, val);
    return;
  }
  const size_t vb = 3 * (size_t)r[RB_V + (q - 9)];
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

// One tile with its top-left pixel (x0, y0).  Entered and left with a clear
// hash table (bwd_clear once per CTA before the first tile); blockDim.x must
// be BWD_THREADS.  gl* collect this thread's share of dL/dL.
// PERSP: perspective-correct barycentrics (sc.invw set).
template <bool PERSP = false>
__device__ __forceinline__ void backward_tile(const BwdScene& sc, int x0, int y0, BwdSmem& sm, float L0, float L1,
                                              float L2, float& gl0, float& gl1, float& gl2) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int x = x0 + (tid & (BWD_TILE_W - 1)), y = y0 + tid / BWD_TILE_W;  // a warp covers 16 x 2 pixels
  const bool inside = x < sc.W && y < sc.H;
  const size_t o = (size_t)y * sc.W + x;
  unsigned t = BWD_NONE;
  if (inside) {
    const unsigned long long k = __ldg(sc.key + o);
    // a key naming a triangle outside this scene contributes nothing (it
    // cannot come from this scene's forward)
    if (k != KEY_EMPTY && (unsigned)k < (unsigned)sc.T) t = (unsigned)k;
  }
  // 1. distinct triangles into the hash table (empty on entry)
  const unsigned grp = __match_any_sync(FULL_MASK, t);
  const int leader = __ffs(grp) - 1;
  int h = 0;
  if (t != BWD_NONE && lane == leader) {
    h = (int)((t * 2654435761u) >> (32 - BWD_HASH_BITS));
    // at most BWD_THREADS keys in BWD_HASH entries: a free or equal entry
    // is always found
    for (int probe = 0; probe < BWD_HASH; ++probe) {
      const unsigned old = atomicCAS(&sm.hkey[h], BWD_NONE, t);
      if (old == BWD_NONE || old == t) break;
      h = (h + 1) & (BWD_HASH - 1);
    }
  }
  // the inserts are complete after this barrier; with nothing visible the
  // table stayed clear and the tile is done
  if (!__syncthreads_or(t != BWD_NONE)) return;
  // 2. slots for the occupied entries; one setup per slot
  for (int e = tid; e < BWD_HASH; e += BWD_THREADS) {
    const unsigned key = sm.hkey[e];
    if (key != BWD_NONE) {
      const int s = atomicAdd(&sm.nslot, 1);
      sm.hslot[e] = (unsigned short)s;
      sm.rec[s * BWD_REC + RB_T] = (int)key;
    }
  }
  __syncthreads();
  const int nslot = sm.nslot;
  const bool direct = nslot > BWD_DIRECT_SLOTS;
  for (int s = tid; s < nslot; s += BWD_THREADS) {
    int* r = sm.rec + s * BWD_REC;
    const unsigned tri = (unsigned)r[RB_T];
    const int ia = __ldg(sc.tris + 3 * (size_t)tri), ib = __ldg(sc.tris + 3 * (size_t)tri + 1),
              ic = __ldg(sc.tris + 3 * (size_t)tri + 2);
    TriSetup ts;
    const bool in_range = ia >= 0 && ia < sc.V && ib >= 0 && ib < sc.V && ic >= 0 && ic < sc.V;
    const bool ok = in_range && setup_triangle(ia, ib, ic, sc.vtx, ts);
    // a winner the vertex stage rejected was clipped: per-pixel ray weights (2)
    const bool clipped = !ok && in_range && sc.pos;
    r[RB_OK] = ok ? 1 : (clipped ? 2 : 0);
    if (clipped) {
      ts.v0 = ia; ts.v1 = ib; ts.v2 = ic;
      r[RB_V] = ia; r[RB_V + 1] = ib; r[RB_V + 2] = ic;
      if (sc.mode == PIKO_SHADE_LAMBERT) {
        const int vid[3] = {ia, ib, ic};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float* nn = sc.normal + 3 * (size_t)vid[j];
          r[RB_VD + j] = __float_as_int(__ldg(nn) * L0 + __ldg(nn + 1) * L1 + __ldg(nn + 2) * L2);
        }
      }
    }
    if (ok) {
      r[0] = ts.X0; r[1] = ts.Y0; r[2] = ts.X1; r[3] = ts.Y1; r[4] = ts.X2; r[5] = ts.Y2;
      r[RB_V] = ts.v0; r[RB_V + 1] = ts.v1; r[RB_V + 2] = ts.v2;
      r[RB_ALO] = (int)(unsigned)(ts.A & 0xFFFFFFFFll);
      r[RB_AHI] = (int)(ts.A >> 32);
      r[RB_T] = __float_as_int(__frcp_rn(f32_from_i64(ts.A)));
      if (sc.mode == PIKO_SHADE_LAMBERT) {
        const int vid[3] = {ts.v0, ts.v1, ts.v2};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float* nn = sc.normal + 3 * (size_t)vid[j];
          r[RB_VD + j] = __float_as_int(__ldg(nn) * L0 + __ldg(nn + 1) * L1 + __ldg(nn + 2) * L2);
        }
      }
    }
    if (!direct) {
      float* a = sm.acc + s * BWD_VALS;
#pragma unroll
      for (int q = 0; q < BWD_VALS; ++q) a[q] = 0.f;
    }
  }
  const int hl = __shfl_sync(FULL_MASK, h, leader);
  const int slot = t != BWD_NONE ? (int)sm.hslot[hl] : -1;
  __syncthreads();
  // 3. per-pixel terms
  float v[BWD_VALS];
#pragma unroll
  for (int q = 0; q < BWD_VALS; ++q) v[q] = 0.f;
  bool hit = false;
  const int* r = sm.rec + (slot >= 0 ? slot : 0) * BWD_REC;
  if (slot >= 0 && r[RB_OK]) {
    hit = true;
    const int X0 = r[0], Y0 = r[1], X1 = r[2], Y1 = r[3], X2 = r[4], Y2 = r[5];
    const long long A = (long long)(((unsigned long long)(unsigned)r[RB_AHI] << 32) | (unsigned)r[RB_ALO]);
    const int vid[3] = {r[RB_V], r[RB_V + 1], r[RB_V + 2]};
    const float rA = __int_as_float(r[RB_T]);
    float b[3];
    if (r[RB_OK] == 2) {
      clip_ray_weights(sc.pos, sc.mvp, sc.W, sc.H, vid, x, y, b[0], b[1], b[2]);
    } else if (A < (1LL << 31)) {
      // the pixel is covered: its edge functions lie in [0, A], exact in wrapping 32-bit arithmetic
      const int Px = 256 * x + 128, Py = 256 * y + 128;
      const int w1 = edge_fn_wrap32(X2, Y2, X0, Y0, Px, Py), w2 = edge_fn_wrap32(X0, Y0, X1, Y1, Px, Py);
      const int w0 = (int)A - w1 - w2;  // the three edge functions sum to A
      b[0] = (float)w0 * rA; b[1] = (float)w1 * rA; b[2] = (float)w2 * rA;
    } else {
      const long long Px = 256LL * x + 128, Py = 256LL * y + 128;
      const long long w1 = (long long)(X0 - X2) * (Py - Y2) - (long long)(Y0 - Y2) * (Px - X2);
      const long long w2 = (long long)(X1 - X0) * (Py - Y0) - (long long)(Y1 - Y0) * (Px - X0);
      const long long w0 = A - w1 - w2;
      b[0] = f32_from_i64(w0) * rA; b[1] = f32_from_i64(w1) * rA; b[2] = f32_from_i64(w2) * rA;
    }
    if (PERSP && r[RB_OK] == 1)
      perspective_bary(b[0], b[1], b[2], __ldg(sc.invw + vid[0]), __ldg(sc.invw + vid[1]), __ldg(sc.invw + vid[2]));
    const float4 g = __ldg(sc.dl + o);
    if (sc.mode == PIKO_SHADE_GOURAUD) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        v[3 * j] = g.x * b[j]; v[3 * j + 1] = g.y * b[j]; v[3 * j + 2] = g.z * b[j];
      }
    } else {
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
      const float d = b[0] * __int_as_float(r[RB_VD]) + b[1] * __int_as_float(r[RB_VD + 1]) +
                      b[2] * __int_as_float(r[RB_VD + 2]);
      const bool active = sc.unclamped || d > 0.f;
      const float sh = sc.unclamped ? d : fmaxf(d, 0.f);
      const float G = active ? (g.x * a0 + g.y * a1 + g.z * a2) : 0.f;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (sc.color) {
          v[3 * j] = g.x * sh * b[j]; v[3 * j + 1] = g.y * sh * b[j]; v[3 * j + 2] = g.z * sh * b[j];
        }
        v[9 + j] = G * b[j];
      }
    }
  }
  const bool has_c = sc.dcolor != nullptr && (sc.mode == PIKO_SHADE_GOURAUD || sc.color != nullptr);
  const bool has_n = sc.dnormal != nullptr && sc.mode == PIKO_SHADE_LAMBERT;
  const bool has_l = sc.dlight != nullptr && sc.mode == PIKO_SHADE_LAMBERT;
  // 4. Lanes of a group of at most two add their own terms (to the slot's
  // accumulators, or straight to the gradients in direct tiles).  Larger
  // groups are summed term by term first: lane q adds term q over the group.
  const unsigned gsize = hit ? (unsigned)__popc(grp) : 0u;
  if (__reduce_max_sync(FULL_MASK, gsize) <= 2u) {
    if (hit) {
      if (direct) {
#pragma unroll
        for (int q = 0; q < BWD_VALS; ++q)
          if (v[q] != 0.f) bwd_add_term(sc, r, q, v[q], has_c, has_n, has_l, L0, L1, L2, gl0, gl1, gl2);
      } else {
        float* a = sm.acc + slot * BWD_VALS;
#pragma unroll
        for (int q = 0; q < BWD_VALS; ++q) atomicAdd(a + q, v[q]);
      }
    }
  } else {
#pragma unroll
    for (int q = 0; q < BWD_VALS; ++q) sm.stage[warp][q][lane] = v[q];
    __syncwarp();
    unsigned todo = __ballot_sync(FULL_MASK, hit);
    // every round removes at least the round's leader lane
    for (int round = 0; todo != 0u && round < 32; ++round) {
      const int ld = __ffs(todo) - 1;
      const unsigned gm = __shfl_sync(FULL_MASK, grp, ld);
      const int gs = __shfl_sync(FULL_MASK, slot, ld);
      todo &= ~gm;
      if (lane < BWD_VALS) {
        float sum = 0.f;
        for (unsigned m = gm; m; m &= m - 1) sum += sm.stage[warp][lane][__ffs(m) - 1];
        if (direct) {
          if (sum != 0.f)
            bwd_add_term(sc, sm.rec + gs * BWD_REC, lane, sum, has_c, has_n, has_l, L0, L1, L2, gl0, gl1, gl2);
        } else {
          atomicAdd(sm.acc + gs * BWD_VALS + lane, sum);
        }
      }
    }
  }
  __syncthreads();
  // 5. one set of gradient atomics per (slot, term); the hash table (no
  // longer read) is cleared for the next tile meanwhile
  if (!direct) {
    for (int idx = tid; idx < nslot * BWD_VALS; idx += BWD_THREADS) {
      const int s = idx / BWD_VALS, q = idx - s * BWD_VALS;
      const int* rs = sm.rec + s * BWD_REC;
      const float val = sm.acc[idx];
      if (rs[RB_OK] && val != 0.f) bwd_add_term(sc, rs, q, val, has_c, has_n, has_l, L0, L1, L2, gl0, gl1, gl2);
    }
  }
  bwd_clear(sm);
  __syncthreads();
}

}  // namespace piko
