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

// BinRect encoding: culled 0xFFFFFFFF; single bin: lo = x | y << 16 | 0x8000,
// hi = slot inside the bin's single-bin part; several bins: lo = x0 | y0 << 16,
// hi = x1 | y1 << 16.  Bin coordinates are below 4096 (width / 8).
constexpr unsigned RECT_CULLED = 0xFFFFFFFFu;
constexpr unsigned RECT_SINGLE = 0x8000u;

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

// Count-pass work for one batch of 32 triangles (one per lane).
__device__ __forceinline__ void count_batch(const RasterGeom& g, int T, int t, int3 idx, const TriVerts& v,
                                            BinRect* __restrict__ rect, unsigned* __restrict__ cnt, int nbins,
                                            DevStatus* st, int stats, int lane, unsigned lt_mask) {
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
  if (t < T) {
    BinRect r;
    if (!valid) {
      r.lo = RECT_CULLED; r.hi = 0u;
    } else if (single) {
      r.lo = (unsigned)bx0 | ((unsigned)by0 << 16) | RECT_SINGLE; r.hi = slot;
    } else {
      r.lo = (unsigned)bx0 | ((unsigned)by0 << 16); r.hi = (unsigned)bx1 | ((unsigned)by1 << 16);
    }
    rect[t] = r;
  }
  const int bw = bx1 - bx0 + 1;
  const int nb = (valid && !single) ? bw * (by1 - by0 + 1) : 0;
  const MultiSpan m = warp_prefix(nb, lane);
  for (int k0 = 0; k0 < m.total; k0 += 32) {
    const int k = k0 + lane;
    const int owner = pair_owner(m.incl, k < m.total ? k : m.total - 1);
    const int ox = __shfl_sync(FULL_MASK, bx0, owner), oy = __shfl_sync(FULL_MASK, by0, owner);
    const int obw = __shfl_sync(FULL_MASK, bw, owner);
    const int first = __shfl_sync(FULL_MASK, m.incl - nb, owner);
    if (k < m.total) atomicAdd(cnt + nbins + pair_bin(g, k, first, ox, oy, obw), 1u);
  }
}

__global__ void __launch_bounds__(256) k_setup_count(RasterGeom g, int T, const int* __restrict__ tris, int V,
                                                     const int4* __restrict__ vtx, BinRect* __restrict__ rect,
                                                     unsigned* __restrict__ cnt, int nbins, DevStatus* st,
                                                     int stats, const int4* __restrict__ clip_tris,
                                                     unsigned clip_cap) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  // the vertex stage does not touch the status word, and everything before
  // it has completed (it is launched without the early-start attribute)
  if (blockIdx.x == 0 && threadIdx.x == 0) st->scan_ticket = 0u;  // the scan runs after this kernel
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
    count_batch(g, TT, t, ia, va, rect, cnt, nbins, st, stats, lane, lt_mask);
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
                        const int4* clip_tris, unsigned clip_cap) {
  static const int per_sm = resident_per_sm(k_setup_count, 256);
  const long long TT = (long long)T + (clip_tris ? clip_cap : 0u);
  int warps = (int)((TT + 31) / 32);
  int blocks = (warps + 7) / 8;
  blocks = blocks < num_sms * per_sm ? blocks : num_sms * per_sm;
  if (blocks < 1) blocks = 1;  // with no triangles the kernel still resets the scan ticket
  launch_pdl(k_setup_count, blocks, 256, 0, s, g, T, tris, V, vtx, rect, bin_count, g.nbx * g.nby, st, stats,
             clip_tris, clip_cap);
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
__device__ __forceinline__ void scatter_batch(const RasterGeom& g, int base, BinRect r, unsigned pos_single,
                                              unsigned* __restrict__ cursor, unsigned* __restrict__ bin_tris,
                                              unsigned long long capacity, int lane) {
  const bool culled = r.lo == RECT_CULLED;
  const bool single = !culled && (r.lo & RECT_SINGLE);
  // positions are below the scanned total, which is at most the capacity;
  // the bound only guards against inconsistent offsets
  if (single && pos_single < capacity) bin_tris[pos_single] = (unsigned)(base + lane);
  const int bx0 = r.lo & 0xFFFF, by0 = r.lo >> 16, bx1 = r.hi & 0xFFFF, by1 = r.hi >> 16;
  const int bw = bx1 - bx0 + 1;
  const int nb = (!culled && !single) ? bw * (by1 - by0 + 1) : 0;
  const MultiSpan m = warp_prefix(nb, lane);
  for (int k0 = 0; k0 < m.total; k0 += 32) {
    const int k = k0 + lane;
    const int owner = pair_owner(m.incl, k < m.total ? k : m.total - 1);
    const int ox = __shfl_sync(FULL_MASK, bx0, owner), oy = __shfl_sync(FULL_MASK, by0, owner);
    const int obw = __shfl_sync(FULL_MASK, bw, owner);
    const int first = __shfl_sync(FULL_MASK, m.incl - nb, owner);
    if (k < m.total) {
      const unsigned pos = atomicAdd(cursor + pair_bin(g, k, first, ox, oy, obw), 1u);
      if (pos < capacity) bin_tris[pos] = (unsigned)(base + owner);
    }
  }
}

// Offset of a single-bin triangle's entry: off[bin] + its slot (0 otherwise).
__device__ __forceinline__ unsigned single_pos(const RasterGeom& g, BinRect r, const unsigned* __restrict__ bin_off) {
  if (r.lo == RECT_CULLED || !(r.lo & RECT_SINGLE)) return 0u;
  const int bin = (int)(r.lo >> 16) * g.nbx + (int)(r.lo & 0x7FFFu);
  return __ldg(bin_off + bin) + r.hi;
}

__global__ void __launch_bounds__(256) k_scatter(RasterGeom g, int T, const BinRect* __restrict__ rect,
                                                 const unsigned* __restrict__ bin_off,
                                                 unsigned* __restrict__ cursor, unsigned* __restrict__ bin_tris,
                                                 unsigned long long capacity, const DevStatus* st,
                                                 const int4* __restrict__ clip_tris, unsigned clip_cap) {
  pdl_wait();  // offsets, cursors and the status of the scan
  pdl_launch_dependents();
  if (st->flags & STATUS_SKIP_MASK) return;
  T = frame_triangles(T, clip_tris, clip_cap, st);
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
    scatter_batch(g, base, ra, pa, cursor, bin_tris, capacity, lane);
    if (hasB) scatter_batch(g, baseB, rb, pb, cursor, bin_tris, capacity, lane);
  }
}

void launch_scatter(const RasterGeom& g, int T, const BinRect* rect, const unsigned* bin_off, unsigned* cursor,
                    unsigned* bin_tris, unsigned long long capacity, DevStatus* st, int num_sms, cudaStream_t s,
                    const int4* clip_tris, unsigned clip_cap) {
  const long long TT = (long long)T + (clip_tris ? clip_cap : 0u);
  if (TT <= 0) return;
  static const int per_sm = resident_per_sm(k_scatter, 256);
  int warps = (int)((TT + 31) / 32);
  int blocks = (warps + 7) / 8;
  blocks = blocks < num_sms * per_sm ? blocks : num_sms * per_sm;
  launch_pdl(k_scatter, blocks, 256, 0, s, g, T, rect, bin_off, cursor, bin_tris, capacity, st, clip_tris,
             clip_cap);
}

}  // namespace piko
