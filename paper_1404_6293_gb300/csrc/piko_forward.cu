// piko_forward.cu -- forward kernels of the binned rasterizer.
//
//   k_vertex       vertex stage: transform, divide, viewport, 16.8 snap (Sec. 7.1, Vertex Shader)
//   k_clip         near/far clipping of the triangles that cross z = -w or z = w (optional)
//   k_setup_count  triangle setup + AssignBin to bounding-box bins, per-bin counts
//                  (AssignToBoundingBox directive, Sec. 4.3; bin lists of Sec. 6)
//   k_scan         exclusive prefix sum of the counts into CSR offsets (the order-preserving
//                  alternative to per-bin atomics that Sec. 6 names)
//   k_scatter      triangle indices into the bin lists
// The per-tile Process stage is in piko_process.cu.

#include "piko_scan.cuh"

namespace piko {

// ======================================================================
// Vertex stage
// ======================================================================
template <bool INVW>
__global__ void __launch_bounds__(256) k_vertex(int W, int H, int V, const float4* __restrict__ pos,
                                                const float* __restrict__ mvp, int4* __restrict__ vtx,
                                                const float* __restrict__ normal, const float* __restrict__ light,
                                                float* __restrict__ vdot, float* __restrict__ invw) {
  pdl_launch_dependents();  // the count pass may be scheduled; it waits for this grid before reading
  __shared__ float m[16];
  const bool has_m = mvp != nullptr;
  if (has_m) {
    if (threadIdx.x < 16) m[threadIdx.x] = mvp[threadIdx.x];
    __syncthreads();
  }
  const float fW = (float)W, fH = (float)H;
  float L0 = 0.f, L1 = 0.f, L2 = 0.f;
  if (vdot) {
    L0 = __ldg(light); L1 = __ldg(light + 1); L2 = __ldg(light + 2);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    if (vdot) vdot[i] = __ldg(normal + 3 * (size_t)i) * L0 + __ldg(normal + 3 * (size_t)i + 1) * L1 +
                        __ldg(normal + 3 * (size_t)i + 2) * L2;
    // one 16-byte load per vertex, coalesced across the warp
    if (INVW) {
      float w;
      vtx[i] = snap_vertex(__ldg(pos + i), has_m ? m : nullptr, fW, fH, &w);
      // 1 / clip w for perspective-correct attributes (unused when w <= 0:
      // the vertex culls every triangle it belongs to)
      invw[i] = w > 0.0f ? __fdiv_rn(1.0f, w) : 0.0f;
    } else {
      vtx[i] = snap_vertex(__ldg(pos + i), has_m ? m : nullptr, fW, fH);
    }
  }
}

void launch_vertex(int W, int H, int V, const float* pos, const float* mvp, int4* vtx, const float* normal,
                   const float* light, float* vdot, float* invw, int num_sms, cudaStream_t s) {
  if (V <= 0) return;
  // one vertex per thread: every load is in flight at once
  (void)num_sms;
  const int blocks = (V + 255) / 256;
  if (invw)
    k_vertex<true><<<blocks, 256, 0, s>>>(W, H, V, reinterpret_cast<const float4*>(pos), mvp, vtx, normal, light, vdot,
                                          invw);
  else
    k_vertex<false><<<blocks, 256, 0, s>>>(W, H, V, reinterpret_cast<const float4*>(pos), mvp, vtx, normal, light,
                                           vdot, nullptr);
}

// ======================================================================
// Near/far clipping (optional).  A triangle with a vertex the vertex stage
// rejected is clipped in clip space against z + w >= 0 and then w - z >= 0
// (Sutherland-Hodgman over its edges in order from vertex 0; the crossing
// point a + t (b - a), t = d_a / (d_a - d_b), every operation rounded, no
// fused multiply-add); the polygon (3 to 5 points) is fanned from its first
// point; each sub-triangle whose points snap inside the guard band (w > 0,
// Z clamped to [0, 2^24 - 1]) is appended to the sub-triangle list with
// the index of its triangle.  The triangle itself stays culled.
// ======================================================================
struct ClipPt {
  float c[4];
};

__device__ __forceinline__ int clip_plane_pts(const ClipPt* in, int n, ClipPt* out, int plane) {
  int m = 0;
  for (int k = 0; k < n; ++k) {
    const ClipPt& a = in[k];
    const ClipPt& b = in[k + 1 < n ? k + 1 : 0];
    const float da = plane == 0 ? __fadd_rn(a.c[2], a.c[3]) : __fsub_rn(a.c[3], a.c[2]);
    const float db = plane == 0 ? __fadd_rn(b.c[2], b.c[3]) : __fsub_rn(b.c[3], b.c[2]);
    const bool ina = da >= 0.0f, inb = db >= 0.0f;
    if (ina) out[m++] = a;
    if (ina != inb) {
      const float t = __fdiv_rn(da, __fsub_rn(da, db));
      ClipPt v;
#pragma unroll
      for (int q = 0; q < 4; ++q) v.c[q] = __fadd_rn(a.c[q], __fmul_rn(t, __fsub_rn(b.c[q], a.c[q])));
      out[m++] = v;
    }
  }
  return m;
}

// divide, viewport and snap of a clipped point: {X, Y, Z, 1}, or false
__device__ __forceinline__ bool snap_clipped(const ClipPt& p, float fW, float fH, int4& o) {
  const float w = p.c[3];
  if (!(w > 0.0f)) return false;
  const float nx = __fdiv_rn(p.c[0], w), ny = __fdiv_rn(p.c[1], w), nz = __fdiv_rn(p.c[2], w);
  const float sx = __fmul_rn(__fadd_rn(__fmul_rn(nx, 0.5f), 0.5f), fW);
  const float sy = __fmul_rn(__fsub_rn(0.5f, __fmul_rn(ny, 0.5f)), fH);
  const float sz = __fmul_rn(__fadd_rn(__fmul_rn(nz, 0.5f), 0.5f), 16777215.0f);
  const float fx = __fmul_rn(sx, 256.0f), fy = __fmul_rn(sy, 256.0f);
  if (!(fabsf(fx) < 8388608.0f && fabsf(fy) < 8388608.0f)) return false;
  float zr = rintf(sz);
  if (!(zr >= 0.0f)) zr = 0.0f;  // NaN, or below the near plane by rounding
  if (zr > 16777215.0f) zr = 16777215.0f;
  o = make_int4(__float2int_rn(fx), __float2int_rn(fy), (int)zr, 1);
  return true;
}

__global__ void __launch_bounds__(256) k_clip(int W, int H, int T, const int* __restrict__ tris, int V,
                                              const float4* __restrict__ pos, const float* __restrict__ mvp,
                                              const int4* __restrict__ vtx, int4* __restrict__ clip_tris,
                                              unsigned* __restrict__ clip_orig, unsigned cap, DevStatus* st) {
  pdl_wait();  // snapped vertices
  pdl_launch_dependents();
  const float fW = (float)W, fH = (float)H;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    const int i0 = __ldg(tris + 3 * (size_t)t), i1 = __ldg(tris + 3 * (size_t)t + 1),
              i2 = __ldg(tris + 3 * (size_t)t + 2);
    if ((unsigned)i0 >= (unsigned)V || (unsigned)i1 >= (unsigned)V || (unsigned)i2 >= (unsigned)V) continue;
    if (__ldg(vtx + i0).w & __ldg(vtx + i1).w & __ldg(vtx + i2).w) continue;  // nothing to clip
    ClipPt p[8], q[8];
    const int id[3] = {i0, i1, i2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 v = __ldg(pos + id[k]);
      if (mvp) {
        p[k].c[0] = mvp_row(mvp + 0, v); p[k].c[1] = mvp_row(mvp + 4, v);
        p[k].c[2] = mvp_row(mvp + 8, v); p[k].c[3] = mvp_row(mvp + 12, v);
      } else {
        p[k].c[0] = v.x; p[k].c[1] = v.y; p[k].c[2] = v.z; p[k].c[3] = v.w;
      }
    }
    int n = clip_plane_pts(p, 3, q, 0);
    n = clip_plane_pts(q, n, p, 1);
    for (int k = 1; k + 1 < n; ++k) {
      int4 a, b, c;
      if (!snap_clipped(p[0], fW, fH, a) || !snap_clipped(p[k], fW, fH, b) || !snap_clipped(p[k + 1], fW, fH, c))
        continue;
      const unsigned slot = atomicAdd(&st->clip_count, 1u);
      if (slot < cap) {
        clip_tris[3 * (size_t)slot] = a;
        clip_tris[3 * (size_t)slot + 1] = b;
        clip_tris[3 * (size_t)slot + 2] = c;
        clip_orig[slot] = (unsigned)t;
      } else {
        record_error(st, PIKO_ERR_OVERFLOW);
      }
    }
  }
}

void launch_clip(int W, int H, int T, const int* tris, int V, const float* pos, const float* mvp, const int4* vtx,
                 int4* clip_tris, unsigned* clip_orig, unsigned cap, DevStatus* st, int num_sms, cudaStream_t s) {
  if (T <= 0) return;
  long long blocks = (T + 255) / 256;
  if (blocks > 8LL * num_sms) blocks = 8LL * num_sms;
  launch_pdl(k_clip, (int)blocks, 256, 0, s, W, H, T, tris, V, reinterpret_cast<const float4*>(pos), mvp, vtx,
             clip_tris, clip_orig, cap, st);
}

// Triangles of the frame: the input ones, then the clipped sub-triangles
// (when clipping is on).  How many sub-triangles there are is known on the
// device only, after the clip pass.
__device__ __forceinline__ int frame_triangles(int T, const int4* clip_tris, unsigned clip_cap, const DevStatus* st) {
  if (!clip_tris) return T;
  const unsigned n = *reinterpret_cast<const volatile unsigned*>(&st->clip_count);
  return T + (int)(n < clip_cap ? n : clip_cap);
}

// ======================================================================
// Index triple of triangle t (zeros past the end).  Lane l of a warp reads
// triangle base + l, so each of the three loads covers one contiguous
// 384-byte span per warp: coalesced without staging.  (Staging the span
// through shared memory with 16-byte loads was measured slower: the
// shared-memory round trip costs more instructions than it saves.)
// ======================================================================
__device__ __forceinline__ int3 load_tri(const int* __restrict__ tris, int T, int t) {
  if (t >= T) return make_int3(0, 0, 0);
  const long long i = 3LL * t;
  return make_int3(__ldg(tris + i), __ldg(tris + i + 1), __ldg(tris + i + 2));
}

// ======================================================================
// Warp-wide expansion of (triangle, bin) pairs for triangles spanning more
// than one bin: lane j owns nb_j pairs; the warp walks all of them 32 at a
// time, each lane finding the owner of its pair by a binary search over the
// inclusive prefix of nb held across the lanes (warp_prefix / pair_owner in
// piko_internal.cuh).
// ======================================================================
// Bin of pair k of the owner lane's rectangle (x0, y0, width bw; first pair
// index first).
__device__ __forceinline__ int pair_bin(const RasterGeom& g, int k, int first, int x0, int y0, int bw) {
  const int local = k - first;
  const int yy = local / bw;
  return (y0 + yy) * g.nbx + x0 + (local - yy * bw);
}

// Optional exact overlap test of AssignBin (PIKO_OPT_EXACT_BINS): a
// triangle spanning several bins gets an entry in bin b only if none of its
// three edges fails the fill-rule test at every pixel centre of b that lies
// in the triangle's bounding box (the separating-axis test of the triangle
// against that rectangle of centres: its own axes are the bounding box's,
// which the rectangle already lies in).  A dropped bin holds no covered
// sample of the triangle, so the keys do not change; only bin entries of
// large or thin triangles go away.
struct OverlapTri {
  int X0, Y0, X1, Y1, X2, Y2;  // oriented (A > 0)
  int px0, px1, py0, py1;      // pixel centres inside the bounding box, clipped to the screen
};

__device__ __forceinline__ OverlapTri overlap_tri(const RasterGeom& g, int4 p0, int4 p1, int4 p2) {
  const long long A = (long long)(p1.x - p0.x) * (p2.y - p0.y) - (long long)(p2.x - p0.x) * (p1.y - p0.y);
  if (A < 0) {
    const int4 q = p1;
    p1 = p2;
    p2 = q;
  }
  OverlapTri o;
  o.X0 = p0.x; o.Y0 = p0.y; o.X1 = p1.x; o.Y1 = p1.y; o.X2 = p2.x; o.Y2 = p2.y;
  centre_range(min(p0.x, min(p1.x, p2.x)), max(p0.x, max(p1.x, p2.x)), 0, g.W - 1, o.px0, o.px1);
  centre_range(min(p0.y, min(p1.y, p2.y)), max(p0.y, max(p1.y, p2.y)), 0, g.H - 1, o.py0, o.py1);
  return o;
}

// Edge a -> b passes its fill-rule test at some centre of columns [x0, x1] x
// rows [y0, y1]: the edge function (Xb - Xa)(Py - Ya) - (Yb - Ya)(Px - Xa) is
// largest at the corner where -dy (Px) and dx (Py) push it up.
__device__ __forceinline__ bool edge_reaches(int Xa, int Ya, int Xb, int Yb, int x0, int x1, int y0, int y1) {
  const int dx = Xb - Xa, dy = Yb - Ya;
  const int Px = 256 * (dy < 0 ? x1 : x0) + 128, Py = 256 * (dx > 0 ? y1 : y0) + 128;
  return (long long)dx * (Py - Ya) - (long long)dy * (Px - Xa) - (1 - top_left(dx, dy)) >= 0;
}

__device__ __forceinline__ bool overlaps_bin(const RasterGeom& g, const OverlapTri& o, int bx, int by) {
  const int x0 = max(bx << g.bshift_x, o.px0), x1 = min(((bx + 1) << g.bshift_x) - 1, o.px1);
  const int y0 = max(by << g.bshift_y, o.py0), y1 = min(((by + 1) << g.bshift_y) - 1, o.py1);
  return edge_reaches(o.X1, o.Y1, o.X2, o.Y2, x0, x1, y0, y1) && edge_reaches(o.X2, o.Y2, o.X0, o.Y0, x0, x1, y0, y1) &&
         edge_reaches(o.X0, o.Y0, o.X1, o.Y1, x0, x1, y0, y1);
}

// The owner lane's OverlapTri, read by every lane of the warp.
__device__ __forceinline__ OverlapTri shfl_overlap(const OverlapTri& o, int owner) {
  OverlapTri r;
  r.X0 = __shfl_sync(FULL_MASK, o.X0, owner); r.Y0 = __shfl_sync(FULL_MASK, o.Y0, owner);
  r.X1 = __shfl_sync(FULL_MASK, o.X1, owner); r.Y1 = __shfl_sync(FULL_MASK, o.Y1, owner);
  r.X2 = __shfl_sync(FULL_MASK, o.X2, owner); r.Y2 = __shfl_sync(FULL_MASK, o.Y2, owner);
  r.px0 = __shfl_sync(FULL_MASK, o.px0, owner); r.px1 = __shfl_sync(FULL_MASK, o.px1, owner);
  r.py0 = __shfl_sync(FULL_MASK, o.py0, owner); r.py1 = __shfl_sync(FULL_MASK, o.py1, owner);
  return r;
}

// pair_bin's bin coordinates
__device__ __forceinline__ void pair_xy(int k, int first, int x0, int y0, int bw, int& bx, int& by) {
  const int local = k - first;
  const int yy = local / bw;
  by = y0 + yy;
  bx = x0 + (local - yy * bw);
}

// BinRect encoding: culled 0xFFFFFFFF; single bin: lo = x | y << 16 | 0x8000,
// hi = slot inside the bin's single-bin part; several bins: lo = x0 | y0 << 16,
// hi = x1 | y1 << 16.  Bin coordinates are below 4096 (width / 8).
constexpr unsigned RECT_CULLED = 0xFFFFFFFFu;
constexpr unsigned RECT_SINGLE = 0x8000u;

// Heavy triangles of AssignBin: a triangle spanning at least HEAVY_PAIRS
// bins (a quarter-screen triangle spans thousands of 16x16 bins).  The count
// pass walks such a triangle's bins with its whole warp, 32 bins a step,
// with no per-pair owner search.  The scatter pass's cursor atomics return
// a position, so a warp walking thousands of them in a row would be a long
// chain of round trips while the rest of the grid has finished: when the
// handle gives a heavy list, the count pass lists the triangle there as
// chunks of HEAVY_CHUNK pairs and marks its rectangle RECT_HEAVY (bit 31 of
// hi; bin coordinates are below 4096), and the scatter pass's CTAs take the
// chunks after their own triangles, a pair per thread.  A list that is full leaves the
// triangle's entries to its warp.
constexpr int HEAVY_PAIRS = 256;
constexpr int HEAVY_CHUNK = 256;
constexpr unsigned RECT_HEAVY = 0x80000000u;
constexpr unsigned HEAVY_NONE = 0xFFFFFFFFu;  // a chunk slot of a triangle that did not fit

// Read after the grid dependency wait: the count pass that wrote it has
// completed, so a plain (read-only path) load sees its final value.
__device__ __forceinline__ unsigned heavy_count(const DevStatus* st, unsigned epoch, unsigned cap) {
  const unsigned n = __ldg(&st->heavy_n[epoch & 1u]);
  return n < cap ? n : cap;
}

// The vertices of triangle t (an input triangle, or clipped sub-triangle t - T).
__device__ __forceinline__ void tri_points(int T, int t, const int* __restrict__ tris, int V,
                                           const int4* __restrict__ vtx, const int4* __restrict__ clip_tris,
                                           int4& p0, int4& p1, int4& p2, bool& ok) {
  ok = true;
  if (t < T) {
    const int3 i = load_tri(tris, T, t);
    if ((unsigned)i.x >= (unsigned)V || (unsigned)i.y >= (unsigned)V || (unsigned)i.z >= (unsigned)V) {
      ok = false;
      p0 = p1 = p2 = make_int4(0, 0, 0, 0);
      return;
    }
    p0 = __ldg(vtx + i.x); p1 = __ldg(vtx + i.y); p2 = __ldg(vtx + i.z);
  } else {
    const int4* c = clip_tris + 3 * (size_t)(t - T);
    p0 = c[0]; p1 = c[1]; p2 = c[2];
  }
}

// Bin of pair k of a multi-bin rectangle.
__device__ __forceinline__ void rect_pair(BinRect r, int k, int& bx, int& by, int& nb) {
  const int bx0 = r.lo & 0xFFFF, by0 = r.lo >> 16, bx1 = r.hi & 0xFFFF, by1 = (r.hi >> 16) & 0x7FFF;
  const int bw = bx1 - bx0 + 1;
  nb = bw * (by1 - by0 + 1);
  const int yy = k / bw;
  by = by0 + yy;
  bx = bx0 + (k - yy * bw);
}

// ======================================================================
// Scan: one CTA per chunk of SCAN_CHUNK bins (scan_chunk in piko_scan.cuh).
// ======================================================================
constexpr int SCAN_THREADS = FWD_SCAN_THREADS;
constexpr int SCAN_CHUNK = FWD_SCAN_CHUNK;

__global__ void __launch_bounds__(SCAN_THREADS) k_scan(int nbins, unsigned* __restrict__ cnt,
                                                       unsigned* __restrict__ bin_off, unsigned* __restrict__ cursor,
                                                       unsigned long long capacity, DevStatus* st,
                                                       unsigned long long* __restrict__ chunk_state, unsigned epoch,
                                                       long long wait_budget, int withhold) {
  __shared__ ScanSmem sm;
  pdl_wait();  // counts and the ticket reset of the count pass
  pdl_launch_dependents();
  if (threadIdx.x == 0) sm.chunk = (int)atomicAdd(&st->scan_ticket, 1u);
  __syncthreads();
  const int chunk = sm.chunk;
  const int nchunks = (nbins + SCAN_CHUNK - 1) / SCAN_CHUNK;
  if (chunk >= nchunks) return;  // only with a corrupted ticket; the count pass resets it every frame
  scan_chunk(chunk, nchunks, nbins, cnt, bin_off, cursor, capacity, st, chunk_state, epoch, sm, &st->queue_head,
             wait_budget, withhold);
  // one CTA per chunk: every ticket was taken before the last chunk's
  // look-back ended, so the last chunk may reset the ticket
  if (chunk == nchunks - 1 && threadIdx.x == 0) st->scan_ticket = 0u;
}

int scan_chunks(int nbins) { return (nbins + SCAN_CHUNK - 1) / SCAN_CHUNK; }

// ======================================================================
// AssignBin, pass 1: setup + counts.  Counts live in two arrays: entries of
// triangles covering one bin (cnt[b]) and of triangles covering several
// (cnt[nbins + b]).  A single-bin triangle gets its slot here from one atomic
// per group of lanes sharing the bin (__match_any_sync), so the scatter
// needs no atomic for it; multi-bin pairs are spread over the warp.
// ======================================================================
// Vertex data of one triangle, gathered before any of it is used.
struct TriVerts {
  int4 p0, p1, p2;
  bool in_range;
};

__device__ __forceinline__ TriVerts gather_verts(int3 idx, int V, const int4* __restrict__ vtx, bool live) {
  TriVerts v;
  v.in_range = live && (unsigned)idx.x < (unsigned)V && (unsigned)idx.y < (unsigned)V && (unsigned)idx.z < (unsigned)V;
  if (v.in_range) {
    v.p0 = __ldg(vtx + idx.x); v.p1 = __ldg(vtx + idx.y); v.p2 = __ldg(vtx + idx.z);
  } else {
    v.p0 = v.p1 = v.p2 = make_int4(0, 0, 0, 0);
  }
  return v;
}

// Count-pass work for one batch of 32 triangles (one per lane).  EXACT:
// multi-bin pairs pass the exact overlap test first.
template <bool EXACT>
__device__ __forceinline__ void count_batch(const RasterGeom& g, int T, int t, int3 idx, const TriVerts& v,
                                            BinRect* __restrict__ rect, unsigned* __restrict__ cnt, int nbins,
                                            DevStatus* st, int stats, int lane, unsigned lt_mask,
                                            uint2* __restrict__ heavy, unsigned heavy_cap, unsigned* heavy_n) {
  bool valid = false;
  int bx0 = 0, by0 = 0, bx1 = -1, by1 = -1;
  if (t < T) {
    if (!v.in_range) {
      record_error(st, PIKO_ERR_BAD_INDEX);
    } else if (v.p0.w & v.p1.w & v.p2.w) {
      const long long A = (long long)(v.p1.x - v.p0.x) * (v.p2.y - v.p0.y) -
                          (long long)(v.p2.x - v.p0.x) * (v.p1.y - v.p0.y);
      if (A != 0) {
        int px0, px1, py0, py1;
        centre_range(min(v.p0.x, min(v.p1.x, v.p2.x)), max(v.p0.x, max(v.p1.x, v.p2.x)), 0, g.W - 1, px0, px1);
        centre_range(min(v.p0.y, min(v.p1.y, v.p2.y)), max(v.p0.y, max(v.p1.y, v.p2.y)), 0, g.H - 1, py0, py1);
        if (px0 <= px1 && py0 <= py1) {  // some pixel centre inside the bounding box
          valid = true;
          bx0 = px0 >> g.bshift_x; bx1 = px1 >> g.bshift_x;
          by0 = py0 >> g.bshift_y; by1 = py1 >> g.bshift_y;
        }
      }
    }
  }
  (void)idx;
  if (stats) {
    const unsigned nv = __popc(__ballot_sync(FULL_MASK, valid));
    if (lane == 0 && nv) atomicAdd(&st->binned, (unsigned long long)nv);
  }
  const bool single = valid && bx0 == bx1 && by0 == by1;
  const unsigned bin = single ? (unsigned)(by0 * g.nbx + bx0) : 0xFFFFFFFFu;
  const unsigned grp = __match_any_sync(FULL_MASK, bin);
  const int leader = __ffs(grp) - 1;
  unsigned slot = 0;
  if (single && lane == leader) slot = atomicAdd(cnt + bin, (unsigned)__popc(grp));
  slot = __shfl_sync(FULL_MASK, slot, leader) + __popc(grp & lt_mask);
  const int bw = bx1 - bx0 + 1;
  int nb = (valid && !single) ? bw * (by1 - by0 + 1) : 0;
  bool listed = false;
  OverlapTri ot;
  if (EXACT && __any_sync(FULL_MASK, nb > 0)) ot = overlap_tri(g, v.p0, v.p1, v.p2);
  // heavy triangles, one at a time: the whole warp walks its bins 32 at a
  // time (no owner search), each lane stepping 32 bins along the rectangle
  for (unsigned hv = __ballot_sync(FULL_MASK, nb >= HEAVY_PAIRS); hv != 0u; hv &= hv - 1u) {
    const int owner = __ffs(hv) - 1;
    const int hx0 = __shfl_sync(FULL_MASK, bx0, owner), hy0 = __shfl_sync(FULL_MASK, by0, owner);
    const int hbw = __shfl_sync(FULL_MASK, bw, owner), hnb = __shfl_sync(FULL_MASK, nb, owner);
    OverlapTri o;
    if (EXACT) o = shfl_overlap(ot, owner);
    const int sy = 32 / hbw, sx = 32 - sy * hbw;
    int lx = lane % hbw, ly = lane / hbw;
    for (int k = lane; k < hnb; k += 32) {
      if (!EXACT || overlaps_bin(g, o, hx0 + lx, hy0 + ly)) atomicAdd(cnt + nbins + (hy0 + ly) * g.nbx + hx0 + lx, 1u);
      lx += sx; ly += sy;
      if (lx >= hbw) { lx -= hbw; ++ly; }
    }
  }
  const bool heavy_tri = nb >= HEAVY_PAIRS;
  if (heavy && heavy_tri) {
    const unsigned nch = (unsigned)((nb + HEAVY_CHUNK - 1) / HEAVY_CHUNK);
    const unsigned pos = atomicAdd(heavy_n, nch);
    listed = pos < heavy_cap && nch <= heavy_cap - pos;
    for (unsigned c = 0; c < nch && pos + c < heavy_cap; ++c)
      heavy[pos + c] = make_uint2(listed ? (unsigned)t : HEAVY_NONE, c);
  }
  if (heavy_tri) nb = 0;  // counted above
  if (t < T) {
    BinRect r;
    if (!valid) {
      r.lo = RECT_CULLED; r.hi = 0u;
    } else if (single) {
      r.lo = (unsigned)bx0 | ((unsigned)by0 << 16) | RECT_SINGLE; r.hi = slot;
    } else {
      r.lo = (unsigned)bx0 | ((unsigned)by0 << 16);
      r.hi = (unsigned)bx1 | ((unsigned)by1 << 16) | (listed ? RECT_HEAVY : 0u);
    }
    rect[t] = r;
  }
  const MultiSpan m = warp_prefix(nb, lane);
  for (int k0 = 0; k0 < m.total; k0 += 32) {
    const int k = k0 + lane;
    const int owner = pair_owner(m.incl, k < m.total ? k : m.total - 1);
    const int ox = __shfl_sync(FULL_MASK, bx0, owner), oy = __shfl_sync(FULL_MASK, by0, owner);
    const int obw = __shfl_sync(FULL_MASK, bw, owner);
    const int first = __shfl_sync(FULL_MASK, m.incl - nb, owner);
    if (EXACT) {
      const OverlapTri o = shfl_overlap(ot, owner);
      int bx, by;
      pair_xy(k, first, ox, oy, obw, bx, by);
      if (k < m.total && overlaps_bin(g, o, bx, by)) atomicAdd(cnt + nbins + by * g.nbx + bx, 1u);
    } else if (k < m.total) {
      atomicAdd(cnt + nbins + pair_bin(g, k, first, ox, oy, obw), 1u);
    }
  }
}

// Scan of a frame of one scan chunk, fused into the count pass (SCAN): the
// count pass's last CTA to finish (each CTA counts itself out after a fence
// that makes its count atomics visible) scans the counts.  No CTA waits for
// another.
struct FusedScan {
  unsigned* bin_off;
  unsigned* cursor;
  unsigned long long capacity;
  unsigned long long* chunk_state;
  unsigned epoch;
};

// eight CTAs of 256 threads per SM (32 registers) for the default binning,
// four (64 registers) with the exact overlap test
template <bool EXACT, bool SCAN = false>
__global__ void __launch_bounds__(256, EXACT ? 4 : 8) k_setup_count(RasterGeom g, int T, const int* __restrict__ tris, int V,
                                                     const int4* __restrict__ vtx, BinRect* __restrict__ rect,
                                                     unsigned* __restrict__ cnt, int nbins, DevStatus* st,
                                                     int stats, const int4* __restrict__ clip_tris,
                                                     unsigned clip_cap, uint2* __restrict__ heavy,
                                                     unsigned heavy_cap, unsigned heavy_epoch, FusedScan fs) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // the vertex stage does not touch the status word, and everything before
  // it has completed (it is launched without the early-start attribute)
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->scan_ticket = 0u;  // the scan runs after this kernel
    // the other parity's heavy counter is the next count pass's: nothing reads it until then
    st->heavy_n[(heavy_epoch + 1u) & 1u] = 0u;
  }
  unsigned* heavy_n = &st->heavy_n[heavy_epoch & 1u];
  pdl_wait();  // snapped vertices
  pdl_launch_dependents();
  const unsigned lt_mask = (1u << lane) - 1u;
  const int step = gridDim.x * (blockDim.x >> 5) * 32;
  // one batch of 32 triangles per warp and iteration: at 28 registers eight
  // CTAs fit an SM, and the other warps hide the gathers' latency (two
  // batches in flight per warp needed 48 registers, five CTAs, and ran 2%
  // slower end to end)
  const int TT = frame_triangles(T, clip_tris, clip_cap, st);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + wib) * 32; base < TT; base += step) {
    const int t = base + lane;
    const int3 ia = load_tri(tris, T, t);
    TriVerts va = gather_verts(ia, V, vtx, t < T);
    if (t >= T && t < TT) {  // a clipped sub-triangle: its snapped points
      const int4* c = clip_tris + 3 * (size_t)(t - T);
      va.p0 = c[0]; va.p1 = c[1]; va.p2 = c[2];
      va.in_range = true;
    }
    count_batch<EXACT>(g, TT, t, ia, va, rect, cnt, nbins, st, stats, lane, lt_mask, heavy, heavy_cap, heavy_n);
  }
  if (SCAN) {
    __shared__ ScanSmem scan_sm;
    __shared__ int s_last;
    __threadfence();  // this thread's count atomics, before the CTA counts itself out
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&st->count_done, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (s_last) {
      __threadfence();
      if (threadIdx.x == 0) st->count_done = 0u;  // for the next frame
      scan_chunk(0, 1, nbins, cnt, fs.bin_off, fs.cursor, fs.capacity, st, fs.chunk_state, fs.epoch, scan_sm,
                 &st->queue_head);
    }
  }
}

// Resident CTAs per SM of a kernel (one wave of a persistent grid).
template <typename K>
static int resident_per_sm(K kernel, int threads) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  return n;
}

void launch_setup_count(const RasterGeom& g, int T, const int* tris, int V, const int4* vtx, BinRect* rect,
                        unsigned* bin_count, DevStatus* st, int stats, int num_sms, cudaStream_t s,
                        const int4* clip_tris, unsigned clip_cap, int exact, uint2* heavy, unsigned heavy_cap,
                        unsigned heavy_epoch) {
  static const int per_sm = resident_per_sm(k_setup_count<false>, 256);
  const long long TT = (long long)T + (clip_tris ? clip_cap : 0u);
  int warps = (int)((TT + 31) / 32);
  int blocks = (warps + 7) / 8;
  blocks = blocks < num_sms * per_sm ? blocks : num_sms * per_sm;
  if (blocks < 1) blocks = 1;  // with no triangles the kernel still resets the scan ticket
  launch_pdl(exact ? k_setup_count<true> : k_setup_count<false>, blocks, 256, 0, s, g, T, tris, V, vtx, rect,
             bin_count, g.nbx * g.nby, st, stats, clip_tris, clip_cap, heavy_cap ? heavy : nullptr, heavy_cap,
             heavy_epoch, FusedScan{});
}

bool launch_count_and_scan(const RasterGeom& g, int T, const int* tris, int V, const int4* vtx, BinRect* rect,
                           unsigned* bin_count, DevStatus* st, int stats, int num_sms, cudaStream_t s,
                           const int4* clip_tris, unsigned clip_cap, int exact, uint2* heavy, unsigned heavy_cap,
                           unsigned heavy_epoch, unsigned* bin_off, unsigned* cursor, unsigned long long capacity,
                           unsigned long long* chunk_state, unsigned scan_epoch) {
  const int nbins = g.nbx * g.nby;
  // one chunk of the count pass's 256 threads x SCAN_PER bins
  if (nbins > 256 * SCAN_PER) return false;
  static const int per_sm = resident_per_sm(k_setup_count<false, true>, 256);
  const long long TT = (long long)T + (clip_tris ? clip_cap : 0u);
  int warps = (int)((TT + 31) / 32);
  int blocks = (warps + 7) / 8;
  blocks = blocks < num_sms * per_sm ? blocks : num_sms * per_sm;
  if (blocks < 1) blocks = 1;  // with no triangles the one CTA still scans (all counts zero)
  FusedScan fs;
  fs.bin_off = bin_off;
  fs.cursor = cursor;
  fs.capacity = capacity;
  fs.chunk_state = chunk_state;
  fs.epoch = scan_epoch;
  launch_pdl(exact ? k_setup_count<true, true> : k_setup_count<false, true>, blocks, 256, 0, s, g, T, tris, V, vtx,
             rect, bin_count, nbins, st, stats, clip_tris, clip_cap, heavy_cap ? heavy : nullptr, heavy_cap,
             heavy_epoch, fs);
  return true;
}

void launch_scan(int nbins, unsigned* bin_count, unsigned* bin_off, unsigned* cursor, unsigned long long capacity,
                 DevStatus* st, unsigned long long* chunk_state, unsigned epoch, cudaStream_t s, long long wait_budget,
                 int withhold) {
  launch_pdl(k_scan, scan_chunks(nbins), SCAN_THREADS, 0, s, nbins, bin_count, bin_off, cursor, capacity, st,
             chunk_state, epoch, wait_budget, withhold);
}

// ======================================================================
// AssignBin, pass 2: scatter triangle indices.  Single-bin triangles write
// at off[bin] + their slot from pass 1; multi-bin pairs take an atomic slot
// after the bin's single-bin part, spread over the warp.
// ======================================================================
// Scatter work for one batch of 32 triangles whose rectangles are loaded.
// EXACT: multi-bin pairs pass the count pass's overlap test; ot is the
// lane's triangle (read only for a multi-bin rectangle).
template <bool EXACT>
__device__ __forceinline__ void scatter_batch(const RasterGeom& g, int base, BinRect r, unsigned pos_single,
                                              unsigned* __restrict__ cursor, unsigned* __restrict__ bin_tris,
                                              unsigned long long capacity, int lane, const OverlapTri& ot) {
  const bool culled = r.lo == RECT_CULLED;
  const bool single = !culled && (r.lo & RECT_SINGLE);
  // positions are below the scanned total, which is at most the capacity;
  // the bound only guards against inconsistent offsets
  if (single && pos_single < capacity) bin_tris[pos_single] = (unsigned)(base + lane);
  const int bx0 = r.lo & 0xFFFF, by0 = r.lo >> 16, bx1 = r.hi & 0xFFFF, by1 = (r.hi >> 16) & 0x7FFF;
  const int bw = bx1 - bx0 + 1;
  // a listed heavy triangle's entries are written from the heavy list
  const int nb = (!culled && !single && !(r.hi & RECT_HEAVY)) ? bw * (by1 - by0 + 1) : 0;
  const MultiSpan m = warp_prefix(nb, lane);
  for (int k0 = 0; k0 < m.total; k0 += 32) {
    const int k = k0 + lane;
    const int owner = pair_owner(m.incl, k < m.total ? k : m.total - 1);
    const int ox = __shfl_sync(FULL_MASK, bx0, owner), oy = __shfl_sync(FULL_MASK, by0, owner);
    const int obw = __shfl_sync(FULL_MASK, bw, owner);
    const int first = __shfl_sync(FULL_MASK, m.incl - nb, owner);
    bool keep = k < m.total;
    if (EXACT) {
      const OverlapTri o = shfl_overlap(ot, owner);
      int bx, by;
      pair_xy(k, first, ox, oy, obw, bx, by);
      keep = keep && overlaps_bin(g, o, bx, by);
    }
    if (keep) {
      const unsigned pos = atomicAdd(cursor + pair_bin(g, k, first, ox, oy, obw), 1u);
      if (pos < capacity) bin_tris[pos] = (unsigned)(base + owner);
    }
  }
}

// The vertices of triangle t for the exact test in the scatter pass (only
// for a multi-bin rectangle: everything else needs none).
__device__ __forceinline__ OverlapTri scatter_overlap(const RasterGeom& g, int T, int t, BinRect r,
                                                      const int* __restrict__ tris, int V,
                                                      const int4* __restrict__ vtx, const int4* __restrict__ clip_tris) {
  OverlapTri o = {};
  if (r.lo == RECT_CULLED || (r.lo & RECT_SINGLE) || (r.hi & RECT_HEAVY)) return o;
  int4 p0, p1, p2;
  if (t < T) {
    const int3 i = load_tri(tris, T, t);
    // a multi-bin rectangle was only written for indices the count pass found in range
    if ((unsigned)i.x >= (unsigned)V || (unsigned)i.y >= (unsigned)V || (unsigned)i.z >= (unsigned)V) return o;
    p0 = __ldg(vtx + i.x); p1 = __ldg(vtx + i.y); p2 = __ldg(vtx + i.z);
  } else {
    const int4* c = clip_tris + 3 * (size_t)(t - T);
    p0 = c[0]; p1 = c[1]; p2 = c[2];
  }
  return overlap_tri(g, p0, p1, p2);
}

// Offset of a single-bin triangle's entry: off[bin] + its slot (0 otherwise).
__device__ __forceinline__ unsigned single_pos(const RasterGeom& g, BinRect r, const unsigned* __restrict__ bin_off) {
  if (r.lo == RECT_CULLED || !(r.lo & RECT_SINGLE)) return 0u;
  const int bin = (int)(r.lo >> 16) * g.nbx + (int)(r.lo & 0x7FFFu);
  return __ldg(bin_off + bin) + r.hi;
}

// eight CTAs of 256 threads per SM (32 registers); the exact test's
// instance keeps its vertices in registers (four CTAs)
template <bool EXACT>
__global__ void __launch_bounds__(256, EXACT ? 4 : 8) k_scatter(RasterGeom g, int T, const BinRect* __restrict__ rect,
                                                 const unsigned* __restrict__ bin_off,
                                                 unsigned* __restrict__ cursor, unsigned* __restrict__ bin_tris,
                                                 unsigned long long capacity, const DevStatus* st,
                                                 const int4* __restrict__ clip_tris, unsigned clip_cap,
                                                 const int* __restrict__ tris, int V, const int4* __restrict__ vtx,
                                                 const uint2* __restrict__ heavy, unsigned heavy_cap,
                                                 unsigned heavy_epoch) {
  pdl_wait();  // offsets, cursors and the status of the scan
  pdl_launch_dependents();
  if (st->flags & STATUS_SKIP_MASK) return;
  const int T_in = T;
  T = frame_triangles(T, clip_tris, clip_cap, st);
  // the heavy list's length is loaded now and used after the per-warp work
  const unsigned nheavy = heavy ? heavy_count(st, heavy_epoch, heavy_cap) : 0u;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int step = gridDim.x * (blockDim.x >> 5) * 32;
  BinRect none;
  none.lo = RECT_CULLED; none.hi = 0u;
  // two batches per iteration, loads first
  for (int base = (blockIdx.x * (blockDim.x >> 5) + wib) * 32; base < T; base += 2 * step) {
    const int baseB = base + step;
    const bool hasB = baseB < T;
    const BinRect ra = base + lane < T ? rect[base + lane] : none;
    const BinRect rb = hasB && baseB + lane < T ? rect[baseB + lane] : none;
    const unsigned pa = single_pos(g, ra, bin_off), pb = single_pos(g, rb, bin_off);
    OverlapTri oa = {}, ob = {};
    if (EXACT) {
      oa = scatter_overlap(g, T_in, base + lane, ra, tris, V, vtx, clip_tris);
      ob = scatter_overlap(g, T_in, baseB + lane, rb, tris, V, vtx, clip_tris);
    }
    scatter_batch<EXACT>(g, base, ra, pa, cursor, bin_tris, capacity, lane, oa);
    if (hasB) scatter_batch<EXACT>(g, baseB, rb, pb, cursor, bin_tris, capacity, lane, ob);
  }
  // the heavy list's chunks, one per CTA step, a pair per thread
  for (unsigned e = blockIdx.x; e < nheavy; e += gridDim.x) {
    const uint2 h = heavy[e];
    if (h.x == HEAVY_NONE || threadIdx.x >= HEAVY_CHUNK) continue;
    const int k = (int)h.y * HEAVY_CHUNK + (int)threadIdx.x;
    int bx, by, nb;
    rect_pair(rect[h.x], k, bx, by, nb);
    if (k >= nb) continue;
    if (EXACT) {
      int4 p0, p1, p2;
      bool ok;
      tri_points(T_in, (int)h.x, tris, V, vtx, clip_tris, p0, p1, p2, ok);
      if (!ok || !overlaps_bin(g, overlap_tri(g, p0, p1, p2), bx, by)) continue;
    }
    const unsigned pos = atomicAdd(cursor + by * g.nbx + bx, 1u);
    if (pos < capacity) bin_tris[pos] = h.x;
  }
}

void launch_scatter(const RasterGeom& g, int T, const BinRect* rect, const unsigned* bin_off, unsigned* cursor,
                    unsigned* bin_tris, unsigned long long capacity, DevStatus* st, int num_sms, cudaStream_t s,
                    const int4* clip_tris, unsigned clip_cap, const int* tris, int V, const int4* vtx,
                    const uint2* heavy, unsigned heavy_cap, unsigned heavy_epoch) {
  const long long TT = (long long)T + (clip_tris ? clip_cap : 0u);
  if (TT <= 0) return;
  static const int per_sm = resident_per_sm(k_scatter<false>, 256);
  int warps = (int)((TT + 31) / 32);
  int blocks = (warps + 7) / 8;
  blocks = blocks < num_sms * per_sm ? blocks : num_sms * per_sm;
  launch_pdl(tris ? k_scatter<true> : k_scatter<false>, blocks, 256, 0, s, g, T, rect, bin_off, cursor, bin_tris,
             capacity, st, clip_tris, clip_cap, tris, V, vtx, heavy_cap ? heavy : nullptr, heavy_cap, heavy_epoch);
}

}  // namespace piko
