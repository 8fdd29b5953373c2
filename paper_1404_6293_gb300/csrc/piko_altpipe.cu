// piko_altpipe.cu -- two other mappings of the raster pipeline onto the GPU,
// for the design-space comparison of Sec. 7.2 of the Piko paper.  Both give
// the same keys and colours as the binned path; only the schedule differs.
//
//  PIKO_SCHED_FUSED: full fusion with no tiling (the FreePipe-style point of
//    Sec. 7.2, a DirectMap over primitives): one pass over the triangles
//    rasterizes each bounding box over the whole screen and takes a 64-bit
//    atomic minimum on the key buffer in global memory; a second pass shades
//    every pixel from its winner.  No bins, no on-chip depth buffer, no
//    load balance beyond one warp per 32 triangles.
//  PIKO_SCHED_UNFUSED: the Baseline pipeline of Sec. 7.1 with every stage
//    its own kernel: the rasterizer emits every covered sample as a fragment
//    into a global buffer, the fragment shader shades every fragment (the
//    forward order: before the depth test), the depth test takes the atomic
//    minimum per pixel, and the composite writes the winning fragment's
//    colour.  The fragment buffer's size is checked like the bin lists'; on
//    an overflow the stages after the rasterizer write nothing (the key
//    buffer is left cleared), and at most 2^32 - 1 fragments are counted.
#include <cooperative_groups.h>

#include "piko_tile.cuh"

namespace cg = cooperative_groups;

namespace piko {

struct AltParams {
  TileScene sc;  // scene and framebuffer (key_out is the global key buffer)
  int T, V;
  DevStatus* st;
  // fragment buffers of the unfused pipeline
  unsigned* frag_pix;
  unsigned long long* frag_key;
  float4* frag_rgba;
  uint2* frag_gn;
  uint2* frag_ga;
  unsigned long long frag_cap;
  unsigned clip_cap;  // capacity of the clipped sub-triangle list (sc.clip_tris)
};

constexpr int ALT_THREADS = 256;
constexpr int ALT_SMALL_PX = 64;  // boxes up to this many pixels: one thread; larger: the whole warp

// Where a covered sample goes: the fused pipeline takes the minimum on the
// key buffer; the unfused one appends a fragment.
template <bool EMIT>
__device__ __forceinline__ void alt_cover(const AltParams& p, unsigned o, unsigned long long k) {
  if (!EMIT) {
    unsigned long long* dst = p.sc.key_out + o;
    if (k < *reinterpret_cast<volatile unsigned long long*>(dst)) atomicMin(dst, k);
    return;
  }
  // one atomic per group of lanes that emit together
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(&p.st->frag_count, g.size());
  base = g.shfl(base, 0) + g.thread_rank();
  if (base < p.frag_cap) {
    p.frag_pix[base] = o;
    p.frag_key[base] = k;
  } else {
    record_error(p.st, PIKO_ERR_OVERFLOW);
  }
}

// One thread walks a box (pixels [px0, px1] x [py0, py1] of the screen).
template <bool EMIT, typename I>
__device__ __forceinline__ void alt_walk(const AltParams& p, const TriSetup& s, unsigned t, int px0, int px1, int py0,
                                         int py1) {
  const Edges<I> e = make_edges<I>(s, px0, py0);
  const float rA = approx_rcp(f32_from_i64(s.A));
  const int W = p.sc.g.W;
  I r0 = e.e0, r1 = e.e1, r2 = e.e2;
  for (int y = py0; y <= py1; ++y) {
    I a0 = r0, a1 = r1, a2 = r2;
    for (int x = px0; x <= px1; ++x) {
      if ((a0 | a1 | a2) >= 0) {
        const unsigned z = depth_of((long long)a1 + e.b1, (long long)a2 + e.b2, s, rA);
        alt_cover<EMIT>(p, (unsigned)(y * W + x), ((unsigned long long)z << 32) | t);
      }
      a0 += e.sx0; a1 += e.sx1; a2 += e.sx2;
    }
    r0 += e.sy0; r1 += e.sy1; r2 += e.sy2;
  }
}

// The warp covers one large box 32 pixels at a time (edge functions of
// each lane's pixel directly from the snapped vertices, in 64 bits).
template <bool EMIT>
__device__ __forceinline__ void alt_warp_box(const AltParams& p, const TriSetup& s, unsigned t, int px0, int px1,
                                             int py0, int py1, int lane) {
  const float rA = approx_rcp(f32_from_i64(s.A));
  const int bw = px1 - px0 + 1;
  const long long n = (long long)bw * (py1 - py0 + 1);
  const int b0 = 1 - top_left(s.X2 - s.X1, s.Y2 - s.Y1);
  const int b1 = 1 - top_left(s.X0 - s.X2, s.Y0 - s.Y2);
  const int b2 = 1 - top_left(s.X1 - s.X0, s.Y1 - s.Y0);
  const int W = p.sc.g.W;
  for (long long base = 0; base < n; base += 32) {
    const long long i = base + lane;
    if (i < n) {
      const int y = py0 + (int)(i / bw), x = px0 + (int)(i % bw);
      const int Px = 256 * x + 128, Py = 256 * y + 128;
      const long long w0 = (long long)(s.X2 - s.X1) * (Py - s.Y1) - (long long)(s.Y2 - s.Y1) * (Px - s.X1);
      const long long w1 = (long long)(s.X0 - s.X2) * (Py - s.Y2) - (long long)(s.Y0 - s.Y2) * (Px - s.X2);
      const long long w2 = (long long)(s.X1 - s.X0) * (Py - s.Y0) - (long long)(s.Y1 - s.Y0) * (Px - s.X0);
      if (((w0 - b0) | (w1 - b1) | (w2 - b2)) >= 0) {
        const unsigned z = depth_of(w1, w2, s, rA);
        alt_cover<EMIT>(p, (unsigned)(y * W + x), ((unsigned long long)z << 32) | t);
      }
    }
  }
}

// Rasterizer over triangles: warp w takes triangles 32 w .. 32 w + 31;
// small boxes one per lane, large ones by the whole warp in turn.
template <bool EMIT>
__global__ void __launch_bounds__(ALT_THREADS) k_alt_raster(const __grid_constant__ AltParams p) {
  const int lane = threadIdx.x & 31;
  const int W = p.sc.g.W, H = p.sc.g.H;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  // the frame's triangles: the input ones, then the clipped sub-triangles
  int TT = p.T;
  if (p.sc.clip_tris) {
    const unsigned n = *reinterpret_cast<const volatile unsigned*>(&p.st->clip_count);
    TT += (int)(n < p.clip_cap ? n : p.clip_cap);
  }
  for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < TT; base += warps_total * 32) {
    const int t = base + lane;
    TriSetup s{};
    bool ok = false, big = false;
    int px0 = 0, px1 = -1, py0 = 0, py1 = -1;
    unsigned key_id = (unsigned)t;
    if (t < TT) {
      bool live;
      if (t >= p.T) {  // a clipped sub-triangle keys with its triangle's index
        const int4* cp = p.sc.clip_tris + 3 * (size_t)(t - p.T);
        live = setup_points(__ldg(cp), __ldg(cp + 1), __ldg(cp + 2), s);
        key_id = __ldg(p.sc.clip_orig + (t - p.T));
      } else {
        const int a = __ldg(p.sc.tris + 3 * (size_t)t), b = __ldg(p.sc.tris + 3 * (size_t)t + 1),
                  c = __ldg(p.sc.tris + 3 * (size_t)t + 2);
        // an index outside [0, V) culls the triangle (the count pass of the
        // binned path reports it; here it is reported too)
        live = (unsigned)a < (unsigned)p.V && (unsigned)b < (unsigned)p.V && (unsigned)c < (unsigned)p.V;
        if (!live) record_error(p.st, PIKO_ERR_BAD_INDEX);
        else live = setup_triangle(a, b, c, p.sc.vtx, s);
      }
      if (live) {
        const int minX = min(s.X0, min(s.X1, s.X2)), maxX = max(s.X0, max(s.X1, s.X2));
        const int minY = min(s.Y0, min(s.Y1, s.Y2)), maxY = max(s.Y0, max(s.Y1, s.Y2));
        centre_range(minX, maxX, 0, W - 1, px0, px1);
        centre_range(minY, maxY, 0, H - 1, py0, py1);
        if (px0 <= px1 && py0 <= py1) {
          ok = true;
          const long long npx = (long long)(px1 - px0 + 1) * (py1 - py0 + 1);
          const bool small32 = maxX - minX < 32768 && maxY - minY < 32768;
          big = npx > ALT_SMALL_PX;
          if (!big) {
            if (small32) alt_walk<EMIT, int>(p, s, key_id, px0, px1, py0, py1);
            else alt_walk<EMIT, long long>(p, s, key_id, px0, px1, py0, py1);
          }
        }
      }
    }
    unsigned m = __ballot_sync(FULL_MASK, ok && big);
    while (m) {
      const int j = __ffs(m) - 1;
      m &= m - 1;
      TriSetup sj;
      sj.X0 = __shfl_sync(FULL_MASK, s.X0, j); sj.Y0 = __shfl_sync(FULL_MASK, s.Y0, j);
      sj.X1 = __shfl_sync(FULL_MASK, s.X1, j); sj.Y1 = __shfl_sync(FULL_MASK, s.Y1, j);
      sj.X2 = __shfl_sync(FULL_MASK, s.X2, j); sj.Y2 = __shfl_sync(FULL_MASK, s.Y2, j);
      sj.Z0 = __shfl_sync(FULL_MASK, s.Z0, j); sj.Z1 = __shfl_sync(FULL_MASK, s.Z1, j);
      sj.Z2 = __shfl_sync(FULL_MASK, s.Z2, j);
      sj.A = __shfl_sync(FULL_MASK, s.A, j);
      sj.v0 = sj.v1 = sj.v2 = 0;
      const int qx0 = __shfl_sync(FULL_MASK, px0, j), qx1 = __shfl_sync(FULL_MASK, px1, j);
      const int qy0 = __shfl_sync(FULL_MASK, py0, j), qy1 = __shfl_sync(FULL_MASK, py1, j);
      const unsigned kid = __shfl_sync(FULL_MASK, key_id, j);
      alt_warp_box<EMIT>(p, sj, kid, qx0, qx1, qy0, qy1, lane);
    }
  }
}

// Fused pipeline, second pass: every pixel shaded from its winner.
template <bool PERSP>
__global__ void __launch_bounds__(ALT_THREADS) k_alt_shade_pixels(const __grid_constant__ AltParams p) {
  const int W = p.sc.g.W;
  const long long n = (long long)W * p.sc.g.H;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
    const unsigned long long k = p.sc.key_out[o];
    if (k == KEY_EMPTY) {
      write_empty(p.sc, (size_t)o);
      continue;
    }
    const int y = (int)(o / W), x = (int)(o - (long long)y * W);
    shade_from_global<PERSP, true>(p.sc, (unsigned)(k & 0xFFFFFFFFu), x, y, (size_t)o);
  }
}

// Unfused pipeline, fragment shader: every fragment, visible or not, shaded
// into the fragment's own colour slot.
template <bool PERSP>
__global__ void __launch_bounds__(ALT_THREADS) k_frag_shade(const __grid_constant__ AltParams p) {
  if (p.st->flags & STATUS_SKIP_MASK) return;  // fragment buffer overflowed: no output
  const unsigned long long n = min((unsigned long long)p.st->frag_count, p.frag_cap);
  TileScene fs = p.sc;  // outputs redirected to the fragment buffers, indexed by fragment
  fs.rgba_out = p.frag_rgba;
  fs.gnorm_out = p.frag_gn;
  fs.galb_out = p.frag_ga;
  const int W = p.sc.g.W;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned o = p.frag_pix[i];
    const int y = (int)(o / (unsigned)W), x = (int)(o - (unsigned)y * (unsigned)W);
    shade_from_global<PERSP, true>(fs, (unsigned)(p.frag_key[i] & 0xFFFFFFFFu), x, y, (size_t)i);
  }
}

// Unfused pipeline, depth test: the per-pixel minimum key over the fragments.
__global__ void __launch_bounds__(ALT_THREADS) k_frag_depth(const __grid_constant__ AltParams p) {
  if (p.st->flags & STATUS_SKIP_MASK) return;  // fragment buffer overflowed: no output
  const unsigned long long n = min((unsigned long long)p.st->frag_count, p.frag_cap);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    atomicMin(p.sc.key_out + p.frag_pix[i], p.frag_key[i]);
}

// Unfused pipeline, composite: the fragment whose key won writes its colour
// (exactly one per covered pixel: a triangle covers a pixel at most once).
__global__ void __launch_bounds__(ALT_THREADS) k_frag_composite(const __grid_constant__ AltParams p) {
  if (p.st->flags & STATUS_SKIP_MASK) return;  // fragment buffer overflowed: no output
  const unsigned long long n = min((unsigned long long)p.st->frag_count, p.frag_cap);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned o = p.frag_pix[i];
    if (p.sc.key_out[o] != p.frag_key[i]) continue;
    if (p.sc.mode == PIKO_SHADE_GBUFFER) {
      p.sc.gnorm_out[o] = p.frag_gn[i];
      p.sc.galb_out[o] = p.frag_ga[i];
    } else if (p.sc.rgba_out) {
      p.sc.rgba_out[o] = p.frag_rgba[i];
    }
  }
}

// Empty pixels of the unfused pipeline: colour (or G-buffer) zero where no
// fragment won.
__global__ void __launch_bounds__(ALT_THREADS) k_alt_clear_empty(const __grid_constant__ AltParams p) {
  if (p.st->flags & STATUS_SKIP_MASK) return;  // fragment buffer overflowed: no output
  const long long n = (long long)p.sc.g.W * p.sc.g.H;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x)
    if (p.sc.key_out[o] == KEY_EMPTY) write_empty(p.sc, (size_t)o);
}

static int alt_grid(long long items, int num_sms) {
  long long g = (items + ALT_THREADS - 1) / ALT_THREADS;
  const long long cap = 8LL * num_sms;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

cudaError_t alt_stage(const AltInputs& in, int stage, bool persp, int num_sms, cudaStream_t s) {
  AltParams p;
  TileScene& sc = p.sc;
  sc.g.W = in.W; sc.g.H = in.H;
  sc.g.bshift_x = sc.g.bshift_y = 0; sc.g.nbx = sc.g.nby = 0;
  sc.mode = in.mode; sc.unclamped = in.unclamped; sc.small_px = 0;
  sc.slot_bits = 0; sc.nslots = 0; sc.rec_stride = 0; sc.tri_base = 0;
  sc.tris = in.tris; sc.vtx = in.vtx; sc.color = in.color; sc.normal = in.normal; sc.light = in.light;
  sc.vdot = nullptr; sc.invw = persp ? in.invw : nullptr;
  sc.T = in.T; sc.clip_tris = in.clip_tris; sc.clip_orig = in.clip_orig;
  sc.pos = in.clip_tris ? reinterpret_cast<const float4*>(in.pos) : nullptr;
  sc.mvp = in.mvp;
  sc.key_out = in.key; sc.rgba_out = in.rgba; sc.gnorm_out = in.gnorm; sc.galb_out = in.galb;
  p.T = in.T; p.V = in.V; p.st = in.st;
  p.frag_pix = in.frag_pix; p.frag_key = in.frag_key; p.frag_rgba = in.frag_rgba;
  p.frag_gn = reinterpret_cast<uint2*>(in.frag_rgba);  // G-buffer mode: two uint2 halves of the same slots
  p.frag_ga = p.frag_gn + (in.frag_rgba ? in.frag_cap : 0);
  p.frag_cap = in.frag_cap;
  p.clip_cap = in.clip_cap;
  const long long npx = (long long)in.W * in.H;
  switch (stage) {
    case ALT_RASTER_MIN:
    case ALT_RASTER_EMIT: {
      if (in.T <= 0) return cudaSuccess;
      long long g = ((in.T + 31) / 32 + (ALT_THREADS / 32) - 1) / (ALT_THREADS / 32);
      if (g > 16LL * num_sms) g = 16LL * num_sms;
      if (in.clip_tris) g += (long long)(in.clip_cap / 32 + 1) / (ALT_THREADS / 32) + 1;
      if (g > 16LL * num_sms) g = 16LL * num_sms;
      if (stage == ALT_RASTER_EMIT) k_alt_raster<true><<<(int)g, ALT_THREADS, 0, s>>>(p);
      else k_alt_raster<false><<<(int)g, ALT_THREADS, 0, s>>>(p);
      break;
    }
    case ALT_SHADE_PIXELS:
      if (persp) k_alt_shade_pixels<true><<<alt_grid(npx, num_sms), ALT_THREADS, 0, s>>>(p);
      else k_alt_shade_pixels<false><<<alt_grid(npx, num_sms), ALT_THREADS, 0, s>>>(p);
      break;
    case ALT_FRAG_SHADE:
      if (persp) k_frag_shade<true><<<alt_grid((long long)in.frag_cap, num_sms), ALT_THREADS, 0, s>>>(p);
      else k_frag_shade<false><<<alt_grid((long long)in.frag_cap, num_sms), ALT_THREADS, 0, s>>>(p);
      break;
    case ALT_FRAG_DEPTH: k_frag_depth<<<alt_grid((long long)in.frag_cap, num_sms), ALT_THREADS, 0, s>>>(p); break;
    case ALT_FRAG_COMPOSITE:
      k_frag_composite<<<alt_grid((long long)in.frag_cap, num_sms), ALT_THREADS, 0, s>>>(p);
      break;
    default: k_alt_clear_empty<<<alt_grid(npx, num_sms), ALT_THREADS, 0, s>>>(p); break;
  }
  return cudaGetLastError();
}

}  // namespace piko
