// piko_forward.cu -- forward kernels of the binned rasterizer.
//
//   k_vertex       vertex stage: transform, divide, viewport, 16.8 snap (Sec. 7.1, Vertex Shader)
//   k_setup_count  triangle setup + AssignBin to bounding-box bins, per-bin counts
//                  (AssignToBoundingBox directive, Sec. 4.3; bin lists of Sec. 6)
//   k_scan         exclusive prefix sum of the counts into CSR offsets (the order-preserving
//                  alternative to per-bin atomics that Sec. 6 names)
//   k_scatter      triangle indices into the bin lists
//   k_process      per-tile Process: coverage, depth test and shading fused (Sec. 5.2.1), with the
//                  tile's depth|ID buffer on chip (Sec. 5.2.4), tiles scheduled statically
//                  (DirectMap), from an atomic queue (LoadBalance) or one CTA per tile.
#include <cuda_fp16.h>

#include "piko_internal.cuh"

namespace piko {

// ======================================================================
// Vertex stage
// ======================================================================
__device__ __forceinline__ float mvp_row(const float* m, float4 p) {
  // ((m0*x + m1*y) + m2*z) + m3*w, every operation rounded, no contraction
  float acc = __fmul_rn(m[0], p.x);
  acc = __fadd_rn(acc, __fmul_rn(m[1], p.y));
  acc = __fadd_rn(acc, __fmul_rn(m[2], p.z));
  acc = __fadd_rn(acc, __fmul_rn(m[3], p.w));
  return acc;
}

__global__ void __launch_bounds__(256) k_vertex(int W, int H, int V, const float4* __restrict__ pos,
                                                const float* __restrict__ mvp, int4* __restrict__ vtx) {
  __shared__ float m[16];
  const bool has_m = mvp != nullptr;
  if (has_m) {
    if (threadIdx.x < 16) m[threadIdx.x] = mvp[threadIdx.x];
    __syncthreads();
  }
  const float fW = (float)W, fH = (float)H;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < V; i += gridDim.x * blockDim.x) {
    const float4 p = __ldg(pos + i);  // one 16-byte load per vertex, coalesced across the warp
    float c0 = p.x, c1 = p.y, c2 = p.z, c3 = p.w;
    if (has_m) {
      c0 = mvp_row(m + 0, p);
      c1 = mvp_row(m + 4, p);
      c2 = mvp_row(m + 8, p);
      c3 = mvp_row(m + 12, p);
    }
    int4 o = make_int4(0, 0, 0, 0);
    if (c3 > 0.0f) {
      const float nx = __fdiv_rn(c0, c3), ny = __fdiv_rn(c1, c3), nz = __fdiv_rn(c2, c3);
      if (nz >= -1.0f && nz <= 1.0f) {
        const float sx = __fmul_rn(__fadd_rn(__fmul_rn(nx, 0.5f), 0.5f), fW);
        const float sy = __fmul_rn(__fsub_rn(0.5f, __fmul_rn(ny, 0.5f)), fH);
        const float sz = __fmul_rn(__fadd_rn(__fmul_rn(nz, 0.5f), 0.5f), 16777215.0f);
        const float fx = __fmul_rn(sx, 256.0f), fy = __fmul_rn(sy, 256.0f);
        if (fabsf(fx) < 8388608.0f && fabsf(fy) < 8388608.0f) {
          o.x = __float2int_rn(fx);
          o.y = __float2int_rn(fy);
          o.z = (int)__float2uint_rn(sz);
          o.w = 1;
        }
      }
    }
    vtx[i] = o;
  }
}

void launch_vertex(int W, int H, int V, const float* pos, const float* mvp, int4* vtx, int num_sms,
                   cudaStream_t s) {
  if (V <= 0) return;
  int blocks = (V + 255) / 256;
  blocks = blocks < num_sms * 8 ? blocks : num_sms * 8;
  k_vertex<<<blocks, 256, 0, s>>>(W, H, V, reinterpret_cast<const float4*>(pos), mvp, vtx);
}

// ======================================================================
// Warp-cooperative, vectorised load of 32 consecutive index triples.
// The warp's 96 indices are read as 24 16-byte loads into a per-warp
// buffer, then each lane takes its own triple.
// ======================================================================
__device__ __forceinline__ int3 load_tri_warp(const int* __restrict__ tris, int T, int base, int lane,
                                              int* __restrict__ wbuf) {
  const long long first = 3LL * base;
  if (base + 32 <= T) {
    if (lane < 24) {
      const int4 q = __ldg(reinterpret_cast<const int4*>(tris + first) + lane);
      reinterpret_cast<int4*>(wbuf)[lane] = q;
    }
  } else {
    const long long n = 3LL * T - first;
    for (int k = lane; k < 96; k += 32) wbuf[k] = k < n ? __ldg(tris + first + k) : 0;
  }
  __syncwarp();
  int3 r = make_int3(wbuf[3 * lane], wbuf[3 * lane + 1], wbuf[3 * lane + 2]);
  __syncwarp();
  return r;
}

// Setup of one triangle for binning: validity and its rectangle of bins.
__device__ __forceinline__ bool bin_setup(const RasterGeom& g, int V, const int4* __restrict__ vtx, int3 idx,
                                          DevStatus* st, int& bx0, int& by0, int& bx1, int& by1) {
  if ((unsigned)idx.x >= (unsigned)V || (unsigned)idx.y >= (unsigned)V || (unsigned)idx.z >= (unsigned)V) {
    record_error(st, PIKO_ERR_BAD_INDEX);
    return false;
  }
  const int4 p0 = __ldg(vtx + idx.x), p1 = __ldg(vtx + idx.y), p2 = __ldg(vtx + idx.z);
  if (!(p0.w & p1.w & p2.w)) return false;
  const long long A = (long long)(p1.x - p0.x) * (long long)(p2.y - p0.y) -
                      (long long)(p2.x - p0.x) * (long long)(p1.y - p0.y);
  if (A == 0) return false;
  int px0, px1, py0, py1;
  centre_range(min(p0.x, min(p1.x, p2.x)), max(p0.x, max(p1.x, p2.x)), 0, g.W - 1, px0, px1);
  centre_range(min(p0.y, min(p1.y, p2.y)), max(p0.y, max(p1.y, p2.y)), 0, g.H - 1, py0, py1);
  if (px0 > px1 || py0 > py1) return false;  // no pixel centre inside the bounding box
  bx0 = px0 >> g.bshift_x; bx1 = px1 >> g.bshift_x;
  by0 = py0 >> g.bshift_y; by1 = py1 >> g.bshift_y;
  return true;
}

// ======================================================================
// AssignBin, pass 1: setup + counts.  Triangles touching one bin (the
// common case for small triangles) are counted with one atomic per group
// of lanes sharing a bin (__match_any_sync); triangles spanning several
// bins are spread over the whole warp, one bin per lane.
// ======================================================================
__global__ void __launch_bounds__(256) k_setup_count(RasterGeom g, int T, const int* __restrict__ tris, int V,
                                                     const int4* __restrict__ vtx, BinRect* __restrict__ rect,
                                                     unsigned* __restrict__ bin_count, DevStatus* st, int stats) {
  __shared__ __align__(16) int sbuf[8][96];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + wib) * 32; base < T; base += warps_total * 32) {
    const int t = base + lane;
    const int3 idx = load_tri_warp(tris, T, base, lane, sbuf[wib]);
    int bx0 = 0, by0 = 0, bx1 = -1, by1 = -1;
    const bool valid = t < T && bin_setup(g, V, vtx, idx, st, bx0, by0, bx1, by1);
    if (t < T) {
      BinRect r;
      r.lo = valid ? ((unsigned)bx0 | ((unsigned)by0 << 16)) : 0xFFFFu;
      r.hi = valid ? ((unsigned)bx1 | ((unsigned)by1 << 16)) : 0u;
      rect[t] = r;
    }
    if (stats) {
      const unsigned nv = __popc(__ballot_sync(FULL_MASK, valid));
      if (lane == 0 && nv) atomicAdd(&st->binned, (unsigned long long)nv);
    }
    const bool single = valid && bx0 == bx1 && by0 == by1;
    const unsigned bin = single ? (unsigned)(by0 * g.nbx + bx0) : 0xFFFFFFFFu;
    const unsigned grp = __match_any_sync(FULL_MASK, bin);
    if (single && lane == __ffs(grp) - 1) atomicAdd(bin_count + bin, (unsigned)__popc(grp));
    unsigned multi = __ballot_sync(FULL_MASK, valid && !single);
    while (multi) {
      const int src = __ffs(multi) - 1;
      multi &= multi - 1;
      const int x0 = __shfl_sync(FULL_MASK, bx0, src), x1 = __shfl_sync(FULL_MASK, bx1, src);
      const int y0 = __shfl_sync(FULL_MASK, by0, src), y1 = __shfl_sync(FULL_MASK, by1, src);
      const int bw = x1 - x0 + 1, nb = bw * (y1 - y0 + 1);
      for (int k = lane; k < nb; k += 32) {
        const int yy = k / bw;
        atomicAdd(bin_count + (y0 + yy) * g.nbx + x0 + (k - yy * bw), 1u);
      }
    }
  }
}

void launch_setup_count(const RasterGeom& g, int T, const int* tris, int V, const int4* vtx, BinRect* rect,
                        unsigned* bin_count, DevStatus* st, int stats, int num_sms, cudaStream_t s) {
  if (T <= 0) return;
  int warps = (T + 31) / 32;
  int blocks = (warps + 7) / 8;
  blocks = blocks < num_sms * 8 ? blocks : num_sms * 8;
  k_setup_count<<<blocks, 256, 0, s>>>(g, T, tris, V, vtx, rect, bin_count, st, stats);
}

// ======================================================================
// Scan: one CTA of 1024 threads, each owning a contiguous run of bins.
// Writes offsets, seeds the scatter cursors with them, zeroes the counts
// for the next frame and records the total (overflow if above capacity).
// ======================================================================
__global__ void __launch_bounds__(1024) k_scan(int nbins, unsigned* __restrict__ bin_count,
                                               unsigned* __restrict__ bin_off, unsigned* __restrict__ cursor,
                                               unsigned long long capacity, DevStatus* st) {
  __shared__ unsigned long long warp_sums[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = (nbins + 1023) / 1024;
  const int b0 = min(tid * per, nbins), b1 = min(b0 + per, nbins);
  unsigned long long local = 0;
  for (int b = b0; b < b1; ++b) local += bin_count[b];
  // inclusive warp scan
  unsigned long long v = local;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(FULL_MASK, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) warp_sums[w] = v;
  __syncthreads();
  if (w == 0) {
    unsigned long long x = warp_sums[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(FULL_MASK, x, o);
      if (lane >= o) x += u;
    }
    warp_sums[lane] = x;  // inclusive over warps
  }
  __syncthreads();
  const unsigned long long total = warp_sums[31];
  unsigned long long run = v - local + (w > 0 ? warp_sums[w - 1] : 0ull);  // exclusive prefix
  const bool ok = total <= capacity;
  for (int b = b0; b < b1; ++b) {
    const unsigned c = bin_count[b];
    bin_count[b] = 0u;
    if (ok) {
      bin_off[b] = (unsigned)run;
      cursor[b] = (unsigned)run;
    }
    run += c;
  }
  if (tid == 0) {
    if (ok) bin_off[nbins] = (unsigned)total;
    st->needed = total;
    st->queue_head = 0u;
    if (!ok) record_error(st, PIKO_ERR_OVERFLOW);
  }
}

void launch_scan(int nbins, unsigned* bin_count, unsigned* bin_off, unsigned* cursor,
                 unsigned long long capacity, DevStatus* st, cudaStream_t s) {
  k_scan<<<1, 1024, 0, s>>>(nbins, bin_count, bin_off, cursor, capacity, st);
}

// ======================================================================
// AssignBin, pass 2: scatter triangle indices.  Single-bin triangles take
// one atomic per group of lanes sharing a bin and write at base + rank.
// ======================================================================
__global__ void __launch_bounds__(256) k_scatter(RasterGeom g, int T, const BinRect* __restrict__ rect,
                                                 unsigned* __restrict__ cursor, unsigned* __restrict__ bin_tris,
                                                 const DevStatus* st) {
  if (st->flags & (1u << PIKO_ERR_OVERFLOW)) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int base = (blockIdx.x * (blockDim.x >> 5) + wib) * 32; base < T; base += warps_total * 32) {
    const int t = base + lane;
    BinRect r;
    r.lo = 0xFFFFu; r.hi = 0u;
    if (t < T) r = rect[t];
    const int bx0 = r.lo & 0xFFFF, by0 = r.lo >> 16, bx1 = r.hi & 0xFFFF, by1 = r.hi >> 16;
    const bool valid = bx0 <= bx1;
    const bool single = valid && bx0 == bx1 && by0 == by1;
    const unsigned bin = single ? (unsigned)(by0 * g.nbx + bx0) : 0xFFFFFFFFu;
    const unsigned grp = __match_any_sync(FULL_MASK, bin);
    if (single) {
      const int leader = __ffs(grp) - 1;
      unsigned slot = 0;
      if (lane == leader) slot = atomicAdd(cursor + bin, (unsigned)__popc(grp));
      slot = __shfl_sync(grp, slot, leader);
      bin_tris[slot + __popc(grp & lt_mask)] = (unsigned)t;
    }
    unsigned multi = __ballot_sync(FULL_MASK, valid && !single);
    while (multi) {
      const int src = __ffs(multi) - 1;
      multi &= multi - 1;
      const int x0 = __shfl_sync(FULL_MASK, bx0, src), x1 = __shfl_sync(FULL_MASK, bx1, src);
      const int y0 = __shfl_sync(FULL_MASK, by0, src), y1 = __shfl_sync(FULL_MASK, by1, src);
      const unsigned tt = (unsigned)(base + src);
      const int bw = x1 - x0 + 1, nb = bw * (y1 - y0 + 1);
      for (int k = lane; k < nb; k += 32) {
        const int yy = k / bw;
        const unsigned slot = atomicAdd(cursor + (y0 + yy) * g.nbx + x0 + (k - yy * bw), 1u);
        bin_tris[slot] = tt;
      }
    }
  }
}

void launch_scatter(const RasterGeom& g, int T, const BinRect* rect, unsigned* cursor, unsigned* bin_tris,
                    DevStatus* st, int num_sms, cudaStream_t s) {
  if (T <= 0) return;
  int warps = (T + 31) / 32;
  int blocks = (warps + 7) / 8;
  blocks = blocks < num_sms * 8 ? blocks : num_sms * 8;
  k_scatter<<<blocks, 256, 0, s>>>(g, T, rect, cursor, bin_tris, st);
}

// ======================================================================
// Process: one tile per CTA iteration.
// ======================================================================
struct EdgeSetup {
  // edge functions minus the fill-rule bias at the first pixel, and their
  // steps per pixel in x and y; covered iff all three are >= 0
  long long e0, e1, e2;
  long long sx0, sx1, sx2, sy0, sy1, sy2;
  int b1, b2;  // bias of edges 1 and 2 (w_i = e_i + b_i)
};

__device__ __forceinline__ void edge_setup(const TriSetup& s, int px, int py, EdgeSetup& e) {
  const long long Px = 256LL * px + 128, Py = 256LL * py + 128;
  // w0 = E_12, w1 = E_20, w2 = E_01 with E_ab(P) = (Xb-Xa)(Py-Ya) - (Yb-Ya)(Px-Xa)
  const int dx0 = s.X2 - s.X1, dy0 = s.Y2 - s.Y1;
  const int dx1 = s.X0 - s.X2, dy1 = s.Y0 - s.Y2;
  const int dx2 = s.X1 - s.X0, dy2 = s.Y1 - s.Y0;
  const int b0 = 1 - top_left(dx0, dy0);
  e.b1 = 1 - top_left(dx1, dy1);
  e.b2 = 1 - top_left(dx2, dy2);
  e.e0 = (long long)dx0 * (Py - s.Y1) - (long long)dy0 * (Px - s.X1) - b0;
  e.e1 = (long long)dx1 * (Py - s.Y2) - (long long)dy1 * (Px - s.X2) - e.b1;
  e.e2 = (long long)dx2 * (Py - s.Y0) - (long long)dy2 * (Px - s.X0) - e.b2;
  e.sx0 = -256LL * dy0; e.sx1 = -256LL * dy1; e.sx2 = -256LL * dy2;
  e.sy0 = 256LL * dx0;  e.sy1 = 256LL * dx1;  e.sy2 = 256LL * dx2;
}

__device__ __forceinline__ void depth_write(unsigned long long* skey, int idx, long long e1, long long e2,
                                            const EdgeSetup& e, const TriSetup& s, float rA, unsigned t) {
  const unsigned z = depth_of(e1 + e.b1, e2 + e.b2, s, rA);
  const unsigned long long k = ((unsigned long long)z << 32) | t;
  if (k < skey[idx]) atomicMin(skey + idx, k);
}

// One thread walks the pixels of a small triangle's box inside the tile.
__device__ __forceinline__ void raster_thread(const TriSetup& s, unsigned t, int px0, int px1, int py0, int py1,
                                              int x0, int y0, int bshift_x, unsigned long long* skey,
                                              unsigned& frags) {
  EdgeSetup e;
  edge_setup(s, px0, py0, e);
  const float rA = __frcp_rn((float)s.A);
  long long r0 = e.e0, r1 = e.e1, r2 = e.e2;
  for (int y = py0; y <= py1; ++y) {
    long long a0 = r0, a1 = r1, a2 = r2;
    const int row = (y - y0) << bshift_x;
    for (int x = px0; x <= px1; ++x) {
      if ((a0 | a1 | a2) >= 0) {
        depth_write(skey, row + (x - x0), a1, a2, e, s, rA, t);
        ++frags;
      }
      a0 += e.sx0; a1 += e.sx1; a2 += e.sx2;
    }
    r0 += e.sy0; r1 += e.sy1; r2 += e.sy2;
  }
}

// A warp covers a large triangle's box 32 pixels at a time; the coverage
// ballot lets the warp skip depth work for fully outside groups.
__device__ __forceinline__ void raster_warp(const TriSetup& s, unsigned t, int px0, int px1, int py0, int py1,
                                            int x0, int y0, int bshift_x, unsigned long long* skey, int lane,
                                            unsigned& frags) {
  EdgeSetup e;
  edge_setup(s, px0, py0, e);
  const float rA = __frcp_rn((float)s.A);
  const int bw = px1 - px0 + 1, n = bw * (py1 - py0 + 1);
  const int dy = 32 / bw, dx = 32 - dy * bw;
  int lx = lane % bw, ly = lane / bw;  // this lane's offset in the box
  for (int base = 0; base < n; base += 32) {
    const bool in_box = base + lane < n;
    const long long a0 = e.e0 + lx * e.sx0 + ly * e.sy0;
    const long long a1 = e.e1 + lx * e.sx1 + ly * e.sy1;
    const long long a2 = e.e2 + lx * e.sx2 + ly * e.sy2;
    const bool cov = in_box && (a0 | a1 | a2) >= 0;
    const unsigned m = __ballot_sync(FULL_MASK, cov);
    if (m != 0u && cov) depth_write(skey, ((py0 + ly - y0) << bshift_x) + (px0 + lx - x0), a1, a2, e, s, rA, t);
    if (lane == 0) frags += __popc(m);
    lx += dx; ly += dy;
    if (lx >= bw) { lx -= bw; ++ly; }
  }
}

__device__ __forceinline__ uint2 pack_half4(float a, float b, float c, float d) {
  const __half2 lo = __floats2half2_rn(a, b), hi = __floats2half2_rn(c, d);
  uint2 r;
  r.x = *reinterpret_cast<const unsigned*>(&lo);
  r.y = *reinterpret_cast<const unsigned*>(&hi);
  return r;
}

// Shading of one pixel from its winning triangle (visibility first: only
// the front-most fragment is shaded; opaque composite keeps no other).
__device__ __forceinline__ void shade_pixel(const ProcessParams& p, int x, int y, unsigned long long k, float L0,
                                            float L1, float L2) {
  const size_t o = (size_t)y * p.g.W + x;
  p.key_out[o] = k;
  if (k == KEY_EMPTY) {
    if (p.mode == PIKO_SHADE_GBUFFER) {
      p.gnorm_out[o] = make_uint2(0u, 0u);
      p.galb_out[o] = make_uint2(0u, 0u);
    } else if (p.rgba_out) {
      p.rgba_out[o] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return;
  }
  const unsigned t = (unsigned)(k & 0xFFFFFFFFu);
  const int a = __ldg(p.tris + 3 * (size_t)t), b = __ldg(p.tris + 3 * (size_t)t + 1),
            c = __ldg(p.tris + 3 * (size_t)t + 2);
  TriSetup s;
  setup_triangle(a, b, c, p.vtx, s);
  const long long Px = 256LL * x + 128, Py = 256LL * y + 128;
  const long long w0 = (long long)(s.X2 - s.X1) * (Py - s.Y1) - (long long)(s.Y2 - s.Y1) * (Px - s.X1);
  const long long w1 = (long long)(s.X0 - s.X2) * (Py - s.Y2) - (long long)(s.Y0 - s.Y2) * (Px - s.X2);
  const long long w2 = (long long)(s.X1 - s.X0) * (Py - s.Y0) - (long long)(s.Y1 - s.Y0) * (Px - s.X0);
  const float fA = (float)s.A;
  const float b0 = __fdiv_rn((float)w0, fA), b1 = __fdiv_rn((float)w1, fA), b2 = __fdiv_rn((float)w2, fA);
  float alb0, alb1, alb2;
  if (p.color) {
    const float* c0 = p.color + 3 * (size_t)s.v0;
    const float* c1 = p.color + 3 * (size_t)s.v1;
    const float* c2 = p.color + 3 * (size_t)s.v2;
    alb0 = b0 * __ldg(c0) + b1 * __ldg(c1) + b2 * __ldg(c2);
    alb1 = b0 * __ldg(c0 + 1) + b1 * __ldg(c1 + 1) + b2 * __ldg(c2 + 1);
    alb2 = b0 * __ldg(c0 + 2) + b1 * __ldg(c1 + 2) + b2 * __ldg(c2 + 2);
  } else {
    alb0 = 0.80f; alb1 = 0.75f; alb2 = 0.65f;  // material of Listing 1
  }
  if (p.mode == PIKO_SHADE_GOURAUD) {
    if (p.rgba_out) p.rgba_out[o] = make_float4(alb0, alb1, alb2, 1.0f);
    return;
  }
  const float* n0 = p.normal + 3 * (size_t)s.v0;
  const float* n1 = p.normal + 3 * (size_t)s.v1;
  const float* n2 = p.normal + 3 * (size_t)s.v2;
  const float nx = b0 * __ldg(n0) + b1 * __ldg(n1) + b2 * __ldg(n2);
  const float ny = b0 * __ldg(n0 + 1) + b1 * __ldg(n1 + 1) + b2 * __ldg(n2 + 1);
  const float nz = b0 * __ldg(n0 + 2) + b1 * __ldg(n1 + 2) + b2 * __ldg(n2 + 2);
  if (p.mode == PIKO_SHADE_GBUFFER) {
    p.gnorm_out[o] = pack_half4(nx, ny, nz, 0.0f);
    p.galb_out[o] = pack_half4(alb0, alb1, alb2, 1.0f);
    return;
  }
  float d = nx * L0 + ny * L1 + nz * L2;
  if (!p.unclamped) d = fmaxf(d, 0.0f);
  if (p.rgba_out) p.rgba_out[o] = make_float4(alb0 * d, alb1 * d, alb2 * d, 1.0f);
}

__global__ void __launch_bounds__(512) k_process(ProcessParams p) {
  extern __shared__ __align__(16) unsigned long long smem[];
  const int bin_w = 1 << p.g.bshift_x, bin_h = 1 << p.g.bshift_y;
  const int bin_px = bin_w * bin_h;
  unsigned long long* skey = smem;
  unsigned* sbig = reinterpret_cast<unsigned*>(smem + bin_px);
  __shared__ int s_tile, s_nbig;
  if (p.st->flags & (1u << PIKO_ERR_OVERFLOW)) return;
  const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  float L0 = 0.f, L1 = 0.f, L2 = 0.f;
  if (p.mode == PIKO_SHADE_LAMBERT) {
    L0 = __ldg(p.light); L1 = __ldg(p.light + 1); L2 = __ldg(p.light + 2);
  }
  unsigned long long n_tests = 0, n_frags = 0, n_shaded = 0;  // PIKO_OPT_STATS only
  for (int iter = 0;; ++iter) {
    int tile;
    if (p.schedule == PIKO_SCHED_HARDWARE) {
      if (iter > 0) break;
      tile = blockIdx.x;
    } else if (p.schedule == PIKO_SCHED_STATIC) {
      tile = blockIdx.x + iter * gridDim.x;
    } else {
      if (tid == 0) s_tile = (int)atomicAdd(&p.st->queue_head, 1u);
      __syncthreads();
      tile = s_tile;
    }
    if (tile >= p.ntiles) break;
    const int tx = tile % p.g.nbx, ty = tile / p.g.nbx;
    const int x0 = tx << p.g.bshift_x, y0 = ty << p.g.bshift_y;
    const int x1 = min(x0 + bin_w, p.g.W) - 1, y1 = min(y0 + bin_h, p.g.H) - 1;
    for (int i = tid; i < bin_px; i += nt) skey[i] = KEY_EMPTY;
    if (tid == 0) s_nbig = 0;
    __syncthreads();
    const unsigned beg = p.bin_off[tile], end = p.bin_off[tile + 1];
    for (unsigned c = beg; c < end; c += nt) {
      const unsigned i = c + tid;
      if (i < end) {
        const unsigned t = __ldg(p.bin_tris + i);
        const int a = __ldg(p.tris + 3 * (size_t)t), b = __ldg(p.tris + 3 * (size_t)t + 1),
                  cc = __ldg(p.tris + 3 * (size_t)t + 2);
        TriSetup s;
        setup_triangle(a, b, cc, p.vtx, s);
        int px0, px1, py0, py1;
        centre_range(min(s.X0, min(s.X1, s.X2)), max(s.X0, max(s.X1, s.X2)), x0, x1, px0, px1);
        centre_range(min(s.Y0, min(s.Y1, s.Y2)), max(s.Y0, max(s.Y1, s.Y2)), y0, y1, py0, py1);
        if (px0 <= px1 && py0 <= py1) {
          const int npx = (px1 - px0 + 1) * (py1 - py0 + 1);
          if (p.stats) n_tests += npx;
          if (npx <= p.small_px) {
            unsigned f = 0;
            raster_thread(s, t, px0, px1, py0, py1, x0, y0, p.g.bshift_x, skey, f);
            if (p.stats) n_frags += f;
          } else {
            sbig[atomicAdd(&s_nbig, 1)] = t;
          }
        }
      }
      __syncthreads();
      const int nbig = s_nbig;
      for (int q = warp; q < nbig; q += nwarps) {
        const unsigned t = sbig[q];
        const int a = __ldg(p.tris + 3 * (size_t)t), b = __ldg(p.tris + 3 * (size_t)t + 1),
                  cc = __ldg(p.tris + 3 * (size_t)t + 2);
        TriSetup s;
        setup_triangle(a, b, cc, p.vtx, s);
        int px0, px1, py0, py1;
        centre_range(min(s.X0, min(s.X1, s.X2)), max(s.X0, max(s.X1, s.X2)), x0, x1, px0, px1);
        centre_range(min(s.Y0, min(s.Y1, s.Y2)), max(s.Y0, max(s.Y1, s.Y2)), y0, y1, py0, py1);
        unsigned f = 0;
        raster_warp(s, t, px0, px1, py0, py1, x0, y0, p.g.bshift_x, skey, lane, f);
        if (p.stats) n_frags += f;
      }
      __syncthreads();
      if (tid == 0) s_nbig = 0;
      __syncthreads();
    }
    // shading and write-out, one thread per pixel, rows contiguous in memory
    for (int i = tid; i < bin_px; i += nt) {
      const int lx = i & (bin_w - 1), ly = i >> p.g.bshift_x;
      const int x = x0 + lx, y = y0 + ly;
      if (x <= x1 && y <= y1) {
        const unsigned long long k = skey[i];
        if (p.stats && k != KEY_EMPTY) ++n_shaded;
        shade_pixel(p, x, y, k, L0, L1, L2);
      }
    }
    __syncthreads();
  }
  if (p.stats) {
    atomicAdd(&p.st->tests, n_tests);
    atomicAdd(&p.st->frags, n_frags);
    atomicAdd(&p.st->shaded, n_shaded);
  }
}

size_t process_smem_bytes(int threads, int bin_px) {
  return (size_t)bin_px * sizeof(unsigned long long) + (size_t)threads * sizeof(unsigned);
}

cudaError_t process_occupancy(int threads, int bin_px, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_process, threads,
                                                       process_smem_bytes(threads, bin_px));
}

cudaError_t launch_process(const ProcessParams& p, int threads, int grid, cudaStream_t s) {
  const int bin_px = 1 << (p.g.bshift_x + p.g.bshift_y);
  k_process<<<grid, threads, process_smem_bytes(threads, bin_px), s>>>(p);
  return cudaGetLastError();
}

}  // namespace piko
