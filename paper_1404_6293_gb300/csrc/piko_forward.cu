// piko_forward.cu -- forward kernels of the binned rasterizer.
//
//   k_vertex       vertex stage: transform, divide, viewport, 16.8 snap (Sec. 7.1, Vertex Shader)
//   k_setup_count  triangle setup + AssignBin to bounding-box bins, per-bin counts
//                  (AssignToBoundingBox directive, Sec. 4.3; bin lists of Sec. 6)
//   k_scan         exclusive prefix sum of the counts into CSR offsets (the order-preserving
//                  alternative to per-bin atomics that Sec. 6 names)
//   k_scatter      triangle indices into the bin lists
// The per-tile Process stage is in piko_process.cu.

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
// Warp-wide expansion of (triangle, bin) pairs for triangles spanning more
// than one bin: lane j owns nb_j pairs; the warp walks all of them 32 at a
// time, each lane finding the owner of its pair by a binary search over the
// inclusive prefix of nb held across the lanes.
// ======================================================================
struct MultiSpan {
  int incl, total;
};

__device__ __forceinline__ MultiSpan warp_prefix(int nb, int lane) {
  int incl = nb;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += u;
  }
  MultiSpan m;
  m.incl = incl;
  m.total = __shfl_sync(FULL_MASK, incl, 31);
  return m;
}

// owner = the smallest lane whose inclusive prefix exceeds k (k < total)
__device__ __forceinline__ int pair_owner(int incl, int k) {
  int owner = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const int v = __shfl_sync(FULL_MASK, incl, owner + s - 1);
    if (v <= k) owner += s;
  }
  return owner;
}

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
// AssignBin, pass 1: setup + counts.  Counts live in two arrays: entries of
// triangles covering one bin (cnt[b]) and of triangles covering several
// (cnt[nbins + b]).  A single-bin triangle gets its slot here from one atomic
// per group of lanes sharing the bin (__match_any_sync), so the scatter
// needs no atomic for it; multi-bin pairs are spread over the warp.
// ======================================================================
__global__ void __launch_bounds__(256) k_setup_count(RasterGeom g, int T, const int* __restrict__ tris, int V,
                                                     const int4* __restrict__ vtx, BinRect* __restrict__ rect,
                                                     unsigned* __restrict__ cnt, int nbins, DevStatus* st,
                                                     int stats) {
  __shared__ __align__(16) int sbuf[8][96];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + wib) * 32; base < T; base += warps_total * 32) {
    const int t = base + lane;
    const int3 idx = load_tri_warp(tris, T, base, lane, sbuf[wib]);
    int bx0 = 0, by0 = 0, bx1 = -1, by1 = -1;
    const bool valid = t < T && bin_setup(g, V, vtx, idx, st, bx0, by0, bx1, by1);
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
}

void launch_setup_count(const RasterGeom& g, int T, const int* tris, int V, const int4* vtx, BinRect* rect,
                        unsigned* bin_count, DevStatus* st, int stats, int num_sms, cudaStream_t s) {
  if (T <= 0) return;
  int warps = (T + 31) / 32;
  int blocks = (warps + 7) / 8;
  blocks = blocks < num_sms * 8 ? blocks : num_sms * 8;
  k_setup_count<<<blocks, 256, 0, s>>>(g, T, tris, V, vtx, rect, bin_count, g.nbx * g.nby, st, stats);
}

// ======================================================================
// Scan: one CTA of 1024 threads walks the bins in rounds of 8192, each
// thread owning 8 consecutive bins (two 16-byte loads per count array).
// off[b] = entries of all earlier bins; the scatter cursor of a bin starts
// after its single-bin part; both count arrays are zeroed for the next frame.
// ======================================================================
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER = 8;

__global__ void __launch_bounds__(SCAN_THREADS) k_scan(int nbins, unsigned* __restrict__ cnt,
                                                       unsigned* __restrict__ bin_off,
                                                       unsigned* __restrict__ cursor, unsigned long long capacity,
                                                       DevStatus* st) {
  __shared__ unsigned long long warp_sums[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  unsigned* __restrict__ multi = cnt + nbins;
  const bool vec = (nbins & 3) == 0;  // 16-byte aligned second array
  unsigned long long carry = 0;
  for (int round = 0; round < nbins; round += SCAN_THREADS * SCAN_PER) {
    const int b0 = round + tid * SCAN_PER;
    unsigned sg[SCAN_PER], mu[SCAN_PER];
    if (vec && b0 + SCAN_PER <= nbins) {
      const uint4 a = *reinterpret_cast<const uint4*>(cnt + b0), b = *reinterpret_cast<const uint4*>(cnt + b0 + 4);
      const uint4 c = *reinterpret_cast<const uint4*>(multi + b0), d = *reinterpret_cast<const uint4*>(multi + b0 + 4);
      sg[0] = a.x; sg[1] = a.y; sg[2] = a.z; sg[3] = a.w; sg[4] = b.x; sg[5] = b.y; sg[6] = b.z; sg[7] = b.w;
      mu[0] = c.x; mu[1] = c.y; mu[2] = c.z; mu[3] = c.w; mu[4] = d.x; mu[5] = d.y; mu[6] = d.z; mu[7] = d.w;
    } else {
#pragma unroll
      for (int j = 0; j < SCAN_PER; ++j) {
        const bool in = b0 + j < nbins;
        sg[j] = in ? cnt[b0 + j] : 0u;
        mu[j] = in ? multi[b0 + j] : 0u;
      }
    }
    unsigned long long local = 0;
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) local += (unsigned long long)sg[j] + mu[j];
    unsigned long long v = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(FULL_MASK, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) warp_sums[w] = v;
    __syncthreads();
    if (w == 0) {
      unsigned long long x = warp_sums[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long u = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= o) x += u;
      }
      warp_sums[lane] = x;
    }
    __syncthreads();
    unsigned long long run = carry + v - local + (w > 0 ? warp_sums[w - 1] : 0ull);
    const unsigned long long round_total = warp_sums[31];
    unsigned of[SCAN_PER], cu[SCAN_PER];
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) {
      of[j] = (unsigned)run;
      cu[j] = (unsigned)(run + sg[j]);
      run += (unsigned long long)sg[j] + mu[j];
    }
    if (vec && b0 + SCAN_PER <= nbins) {
      reinterpret_cast<uint4*>(bin_off + b0)[0] = make_uint4(of[0], of[1], of[2], of[3]);
      reinterpret_cast<uint4*>(bin_off + b0)[1] = make_uint4(of[4], of[5], of[6], of[7]);
      reinterpret_cast<uint4*>(cursor + b0)[0] = make_uint4(cu[0], cu[1], cu[2], cu[3]);
      reinterpret_cast<uint4*>(cursor + b0)[1] = make_uint4(cu[4], cu[5], cu[6], cu[7]);
      const uint4 z = make_uint4(0u, 0u, 0u, 0u);
      reinterpret_cast<uint4*>(cnt + b0)[0] = z;
      reinterpret_cast<uint4*>(cnt + b0)[1] = z;
      reinterpret_cast<uint4*>(multi + b0)[0] = z;
      reinterpret_cast<uint4*>(multi + b0)[1] = z;
    } else {
#pragma unroll
      for (int j = 0; j < SCAN_PER; ++j)
        if (b0 + j < nbins) {
          bin_off[b0 + j] = of[j];
          cursor[b0 + j] = cu[j];
          cnt[b0 + j] = 0u;
          multi[b0 + j] = 0u;
        }
    }
    carry += round_total;
    __syncthreads();  // warp_sums is rewritten by the next round
  }
  if (tid == 0) {
    const bool ok = carry <= capacity;
    if (ok) bin_off[nbins] = (unsigned)carry;
    st->needed = carry;
    st->queue_head = 0u;
    if (!ok) record_error(st, PIKO_ERR_OVERFLOW);
  }
}

void launch_scan(int nbins, unsigned* bin_count, unsigned* bin_off, unsigned* cursor,
                 unsigned long long capacity, DevStatus* st, cudaStream_t s) {
  k_scan<<<1, SCAN_THREADS, 0, s>>>(nbins, bin_count, bin_off, cursor, capacity, st);
}

// ======================================================================
// AssignBin, pass 2: scatter triangle indices.  Single-bin triangles write
// at off[bin] + their slot from pass 1; multi-bin pairs take an atomic slot
// after the bin's single-bin part, spread over the warp.
// ======================================================================
__global__ void __launch_bounds__(256) k_scatter(RasterGeom g, int T, const BinRect* __restrict__ rect,
                                                 const unsigned* __restrict__ bin_off,
                                                 unsigned* __restrict__ cursor, unsigned* __restrict__ bin_tris,
                                                 const DevStatus* st) {
  if (st->flags & (1u << PIKO_ERR_OVERFLOW)) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + wib) * 32; base < T; base += warps_total * 32) {
    const int t = base + lane;
    BinRect r;
    r.lo = RECT_CULLED; r.hi = 0u;
    if (t < T) r = rect[t];
    const bool culled = r.lo == RECT_CULLED;
    const bool single = !culled && (r.lo & RECT_SINGLE);
    if (single) {
      const int bin = (int)(r.lo >> 16) * g.nbx + (int)(r.lo & 0x7FFFu);
      bin_tris[__ldg(bin_off + bin) + r.hi] = (unsigned)t;
    }
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
        bin_tris[pos] = (unsigned)(base + owner);
      }
    }
  }
}

void launch_scatter(const RasterGeom& g, int T, const BinRect* rect, const unsigned* bin_off, unsigned* cursor,
                    unsigned* bin_tris, DevStatus* st, int num_sms, cudaStream_t s) {
  if (T <= 0) return;
  int warps = (T + 31) / 32;
  int blocks = (warps + 7) / 8;
  blocks = blocks < num_sms * 8 ? blocks : num_sms * 8;
  k_scatter<<<blocks, 256, 0, s>>>(g, T, rect, bin_off, cursor, bin_tris, st);
}

}  // namespace piko
