// piko_internal.cuh -- shared declarations of the CUDA rasterizer (not part of the C ABI).
//
// Fixed-point conventions (the library's definition; the paper leaves
// rasterization bits open):
//   16.8 snapped vertex coordinates X, Y (int32, |X| < 2^23), depth Z in
//   [0, 2^24-1]; edge functions in int64; pixel centres at 256*p + 128;
//   key = (z << 32) | triangle index, minimum wins.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/piko_raster.h"

namespace piko {

constexpr unsigned long long KEY_EMPTY = 0xFFFFFFFFFFFFFFFFull;
constexpr unsigned FULL_MASK = 0xFFFFFFFFu;

// Device-side status word, one per handle.
// Programmatic dependent launch (sm_90+).  A kernel launched with
// launch_pdl may start while the kernel before it in the stream is still
// running; it must call pdl_wait() before it reads anything that kernel (or
// an earlier one) writes.  pdl_launch_dependents() lets the next kernel's
// CTAs be scheduled once every CTA of this grid has issued it.  Both are
// no-ops for kernels launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr.val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

struct DevStatus {
  unsigned int flags;           // bit c set when PIKO_ERR c was recorded
  unsigned int first_code;      // first PIKO_ERR_* recorded (0 = none)
  unsigned long long needed;    // bin entries the last scan required
  unsigned int queue_head;      // tile counter of the dynamic schedule
  unsigned int scan_ticket;     // next chunk number of the scan (reset by its last chunk)
  unsigned int frag_count;      // fragments emitted by the unfused pipeline's rasterizer
  unsigned int clip_count;      // sub-triangles appended by the clip pass
  unsigned long long tests;     // statistics (PIKO_OPT_STATS): pixel samples tested
  unsigned long long frags;     // covered samples
  unsigned long long shaded;    // covered pixels after the depth test
  unsigned long long binned;    // triangles that reached at least one bin
  unsigned int heavy_n[2];      // chunks in the heavy-triangle list of AssignBin, by count-pass parity
  unsigned int count_done;      // count-pass CTAs finished (its last CTA scans small frames; then 0 again)
};

// Screen and bin geometry of one framebuffer.
struct RasterGeom {
  int W, H;
  int bshift_x, bshift_y;  // log2 of bin width / height
  int nbx, nby;            // bins per row / column
};

// Per-triangle result of the count pass (encoding in piko_forward.cu).
struct BinRect {
  unsigned int lo, hi;
};

// Conditions after which the bin lists of a frame are not usable.
constexpr unsigned STATUS_SKIP_MASK = (1u << PIKO_ERR_OVERFLOW) | (1u << PIKO_ERR_TIMEOUT);

__device__ __forceinline__ void record_error(DevStatus* st, unsigned code) {
  atomicCAS(&st->first_code, 0u, code);
  atomicOr(&st->flags, 1u << code);
}

// ------------------------------------------------------------- warp spans
// Lane j owns nb_j consecutive items of a warp-wide sequence: the inclusive
// prefix of nb over the lanes, and the total.
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

// owner of item k (k < total) = the smallest lane whose inclusive prefix
// exceeds k: a binary search over the lanes' prefixes (called by all lanes)
__device__ __forceinline__ int pair_owner(int incl, int k) {
  int owner = 0;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const int v = __shfl_sync(FULL_MASK, incl, owner + s - 1);
    if (v <= k) owner += s;
  }
  return owner;
}

// ------------------------------------------------------------------ setup
// Triangle after snapping and orientation: slots 0..2 with A > 0.
struct TriSetup {
  int X0, Y0, X1, Y1, X2, Y2;
  int Z0, Z1, Z2;
  int v0, v1, v2;   // original vertex indices in slot order
  long long A;      // twice the area, 16.8 units squared, > 0
};

// Reads the three snapped vertices of triangle (a, b, c) and orients it.
// Returns false if a vertex was culled by the vertex stage or A == 0.
__device__ __forceinline__ bool setup_triangle(int a, int b, int c, const int4* __restrict__ vtx,
                                               TriSetup& s) {
  const int4 p0 = __ldg(vtx + a), p1 = __ldg(vtx + b), p2 = __ldg(vtx + c);
  if (!(p0.w & p1.w & p2.w)) return false;
  long long A = (long long)(p1.x - p0.x) * (long long)(p2.y - p0.y) -
                (long long)(p2.x - p0.x) * (long long)(p1.y - p0.y);
  if (A == 0) return false;
  s.X0 = p0.x; s.Y0 = p0.y; s.Z0 = p0.z; s.v0 = a;
  if (A > 0) {
    s.X1 = p1.x; s.Y1 = p1.y; s.Z1 = p1.z; s.v1 = b;
    s.X2 = p2.x; s.Y2 = p2.y; s.Z2 = p2.z; s.v2 = c;
    s.A = A;
  } else {
    s.X1 = p2.x; s.Y1 = p2.y; s.Z1 = p2.z; s.v1 = c;
    s.X2 = p1.x; s.Y2 = p1.y; s.Z2 = p1.z; s.v2 = b;
    s.A = -A;
  }
  return true;
}

// Orients a triangle given by three snapped points {X, Y, Z, valid} (a
// clipped sub-triangle); false if A == 0.  Vertex indices are not known.
__device__ __forceinline__ bool setup_points(int4 p0, int4 p1, int4 p2, TriSetup& s) {
  long long A = (long long)(p1.x - p0.x) * (long long)(p2.y - p0.y) -
                (long long)(p2.x - p0.x) * (long long)(p1.y - p0.y);
  s.X0 = p0.x; s.Y0 = p0.y; s.Z0 = p0.z; s.v0 = s.v1 = s.v2 = 0;
  if (A >= 0) {
    s.X1 = p1.x; s.Y1 = p1.y; s.Z1 = p1.z;
    s.X2 = p2.x; s.Y2 = p2.y; s.Z2 = p2.z;
    s.A = A;
  } else {
    s.X1 = p2.x; s.Y1 = p2.y; s.Z1 = p2.z;
    s.X2 = p1.x; s.Y2 = p1.y; s.Z2 = p1.z;
    s.A = -A;
  }
  return A != 0;
}

// Pixel columns / rows whose centres lie inside [min, max] of the snapped
// coordinates, clipped to [lo, hi].  ceil((v-128)/256) and floor((v-128)/256)
// with arithmetic shifts (floor for negatives).
__device__ __forceinline__ void centre_range(int vmin, int vmax, int lo, int hi, int& p0, int& p1) {
  p0 = max((vmin - 128 + 255) >> 8, lo);
  p1 = min((vmax - 128) >> 8, hi);
}

// Edge a->b top-left test in the A > 0, y-down orientation.
__device__ __forceinline__ int top_left(int dx, int dy) { return (dy < 0 || (dy == 0 && dx > 0)) ? 1 : 0; }

// int64 -> float32 on the integer and FP32 pipes.  A plain (float) of a
// 64-bit integer (and a float -> int64 conversion) runs on the FP64 pipe,
// which issues at a small fraction of the FP32 rate on this GPU; the helper
// converts the magnitude's two 32-bit words instead.  Correctly rounded for
// |v| < 2^32 (one rounding); within 2 ulp above that.
__device__ __forceinline__ float f32_from_i64(long long v) {
  const unsigned long long m = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  const float f = __fmaf_rn((float)(unsigned)(m >> 32), 4294967296.0f, (float)(unsigned)(m & 0xFFFFFFFFull));
  return v < 0 ? -f : f;
}

// Edge function of a pixel centre P for edge (a -> b): (Xb - Xa)(Py - Ya) -
// (Yb - Ya)(Px - Xa).  The wrapping 32-bit form is exact whenever the true
// value lies in [-2^31, 2^31), e.g. for a pixel the triangle covers when its
// doubled area A is below 2^31 (then the value lies in [0, A]).
__device__ __forceinline__ int edge_fn_wrap32(int Xa, int Ya, int Xb, int Yb, int Px, int Py) {
  return (int)((unsigned)(Xb - Xa) * (unsigned)(Py - Ya) - (unsigned)(Yb - Ya) * (unsigned)(Px - Xa));
}

// floor(n / A) for A > 0 and |n / A| < 2^25, exact.  The float estimate
// (relative error below 2^-21) is within a few units of the quotient; the
// integer remainder then moves it to the unique q with 0 <= n - q*A < A.
// The fix-up loops run a few times at most for A > 0; their bound only keeps
// inconsistent inputs from spinning.
constexpr int DIV_FIX_LIMIT = 64;

__device__ __forceinline__ long long floor_div_est(long long n, long long A, float rA) {
  long long q = (long long)__float2int_rd(__fmul_rn(f32_from_i64(n), rA));
  long long r = n - q * A;
  for (int it = 0; r < 0 && it < DIV_FIX_LIMIT; ++it) { --q; r += A; }
  for (int it = 0; r >= A && it < DIV_FIX_LIMIT; ++it) { ++q; r -= A; }
  return q;
}

// Same for a 128-bit numerator (huge triangles, A >= 2^38).  The estimate
// comes from the top bits of n; the remainder is kept in 128 bits.
__device__ __forceinline__ long long floor_div_est128(__int128 n, long long A, float rA) {
  const float nf = f32_from_i64((long long)(n >> 32)) * 4294967296.0f + (float)(unsigned)(n & 0xFFFFFFFFu);
  long long q = (long long)__float2int_rd(nf * rA);
  __int128 r = n - (__int128)q * A;
  for (int it = 0; r < 0 && it < DIV_FIX_LIMIT; ++it) { --q; r += A; }
  for (int it = 0; r >= A && it < DIV_FIX_LIMIT; ++it) { ++q; r -= A; }
  return q;
}


// Approximate 1/a (a >= 1): only ever used as an estimate that integer
// arithmetic corrects, or for float barycentrics.
__device__ __forceinline__ float approx_rcp(float a) { return __fdividef(1.0f, a); }

// Depth of a covered sample from its edge functions w1, w2 (w0 = A - w1 - w2):
// z = floor((w0 Z0 + w1 Z1 + w2 Z2) / A) = Z0 + floor((w1 (Z1-Z0) + w2 (Z2-Z0)) / A).
__device__ __forceinline__ unsigned depth_of(long long w1, long long w2, const TriSetup& s, float rA) {
  const long long d1 = (long long)s.Z1 - s.Z0, d2 = (long long)s.Z2 - s.Z0;
  long long q;
  if (s.A < (1LL << 38)) {
    q = floor_div_est(w1 * d1 + w2 * d2, s.A, rA);
  } else {
    q = floor_div_est128((__int128)w1 * d1 + (__int128)w2 * d2, s.A, rA);
  }
  return (unsigned)(s.Z0 + q);
}

// Perspective-correct barycentrics from screen-space ones:
// b'_i = (b_i / w_i) / sum_j (b_j / w_j), given 1/w_i.
__device__ __forceinline__ void perspective_bary(float& b0, float& b1, float& b2, float iw0, float iw1, float iw2) {
  const float q0 = b0 * iw0, q1 = b1 * iw1, q2 = b2 * iw2;
  const float r = __fdiv_rn(1.0f, q0 + q1 + q2);
  b0 = q0 * r;
  b1 = q1 * r;
  b2 = q2 * r;
}

// ------------------------------------------------------------ vertex stage
// ((m0*x + m1*y) + m2*z) + m3*w, every operation rounded, no contraction
__device__ __forceinline__ float mvp_row(const float* m, float4 p) {
  float acc = __fmul_rn(m[0], p.x);
  acc = __fadd_rn(acc, __fmul_rn(m[1], p.y));
  acc = __fadd_rn(acc, __fmul_rn(m[2], p.z));
  acc = __fadd_rn(acc, __fmul_rn(m[3], p.w));
  return acc;
}

// Transform (m may be NULL for the identity), divide, viewport, 16.8 snap:
// {X, Y, Z, 1}, or all zero for a vertex that culls its triangles.  *clip_w
// (when given) receives the clip-space w.
__device__ __forceinline__ int4 snap_vertex(float4 p, const float* m, float fW, float fH, float* clip_w = nullptr) {
  float c0 = p.x, c1 = p.y, c2 = p.z, c3 = p.w;
  if (m) {
    c0 = mvp_row(m + 0, p);
    c1 = mvp_row(m + 4, p);
    c2 = mvp_row(m + 8, p);
    c3 = mvp_row(m + 12, p);
  }
  if (clip_w) *clip_w = c3;
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
  return o;
}

// Weights of a clipped triangle's vertices v[3] at pixel (x, y) of a W x H
// framebuffer: the clip-space weights of the point where the pixel centre's
// ray meets the triangle's plane.  With a_i = X_i - x W_i and c_i = Y_i -
// y W_i (clip coordinates of vertex i from the float32 transform, NDC (x, y)
// of the centre) the weights satisfy a . b = c . b = 0 and sum b = 1, so
// b = (a x c) / sum(a x c).  Float64 (a rare path, and the products cancel).
__device__ __forceinline__ void clip_ray_weights(const float4* pos, const float* mvp, int W, int H, const int v[3],
                                                 int x, int y, float& b0, float& b1, float& b2) {
  const double xn = __dsub_rn(__dmul_rn(__ddiv_rn((double)x + 0.5, (double)W), 2.0), 1.0);
  const double yn = __dsub_rn(1.0, __dmul_rn(__ddiv_rn((double)y + 0.5, (double)H), 2.0));
  double a[3], c[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 q = __ldg(pos + v[k]);
    float cx = q.x, cy = q.y, cw = q.w;
    if (mvp) {
      cx = mvp_row(mvp + 0, q);
      cy = mvp_row(mvp + 4, q);
      cw = mvp_row(mvp + 12, q);
    }
    a[k] = __dsub_rn((double)cx, __dmul_rn(xn, (double)cw));
    c[k] = __dsub_rn((double)cy, __dmul_rn(yn, (double)cw));
  }
  const double n0 = __dsub_rn(__dmul_rn(a[1], c[2]), __dmul_rn(a[2], c[1]));
  const double n1 = __dsub_rn(__dmul_rn(a[2], c[0]), __dmul_rn(a[0], c[2]));
  const double n2 = __dsub_rn(__dmul_rn(a[0], c[1]), __dmul_rn(a[1], c[0]));
  const double sum = __dadd_rn(__dadd_rn(n0, n1), n2);
  if (sum != 0.0) {
    b0 = (float)__ddiv_rn(n0, sum);
    b1 = (float)__ddiv_rn(n1, sum);
    b2 = (float)__ddiv_rn(n2, sum);
  } else {
    b0 = b1 = b2 = 1.0f / 3.0f;
  }
}

// --------------------------------------------------------------- kernels
// Records wanted for a scene whose bin lists hold `entries` entries over
// `tiles` tiles: 1.4 x the mean, in multiples of 32 (1.4 x covers the
// spread of entry counts between tiles of the measured workloads).
inline int slots_for_entries(long long entries, int tiles) {
  if (entries <= 0 || tiles <= 0) return 0;
  const long long want = (14 * entries / tiles + 5 * 32) / (10 * 32) * 32;  // round(1.4 mean / 32) * 32
  return (int)(want < 32 ? 32 : (want > 4096 ? 4096 : want));
}

struct ProcessParams {
  RasterGeom g;
  int ntiles;
  int schedule;
  int small_px;
  int mode;
  int unclamped;
  int slots_hint;  // shading records per tile wanted (0: the largest the key encoding allows)
  int stats;
  int num_triangles;
  int slot_bits;   // set by launch_process: bits of the record slot below the triangle index
  int nslots;      // shared-memory records per tile
  int rec_stride;  // 32-bit words per record
  const int* tris;
  const int4* vtx;
  const float* color;
  const float* normal;
  const float* light;
  const float* vdot;  // n_v . L per vertex (Lambert)
  const float* invw;  // 1 / clip w per vertex: perspective-correct attributes (NULL: screen-space)
  const int4* clip_tris;   // near/far clipping: sub-triangles (NULL: off)
  const unsigned* clip_orig;
  const float* pos;        // the scene's positions and matrix (clipped winners' shading)
  const float* mvp;
  const unsigned* bin_off;
  const unsigned* bin_tris;
  unsigned long long* key_out;
  float4* rgba_out;
  uint2* gnorm_out;  // binary16 x4
  uint2* galb_out;   // binary16 x4
  DevStatus* st;
};

// Vertex stage.  If vdot is not NULL it also stores n_v . L per vertex (the
// Lambert term is linear in the interpolated normal, so per-vertex dots
// interpolate to the same value).
void launch_vertex(int W, int H, int V, const float* pos, const float* mvp, int4* vtx, const float* normal,
                   const float* light, float* vdot, float* invw, int num_sms, cudaStream_t s);
// Count pass and scan (two launches): bin_count holds 2 * nbins counters
// (single-bin and multi-bin entries), zero between frames; the scan turns
// them into CSR offsets and scatter cursors (capacity: entries the bin lists
// can hold; above it PIKO_ERR_OVERFLOW is recorded).
// With clipping, clip_tris / clip_cap describe the sub-triangle list of the
// clip pass (triangles T.. of the frame); otherwise NULL / 0.
// exact: multi-bin triangles get entries only in bins they overlap
// (PIKO_OPT_EXACT_BINS); the scatter pass then needs tris / V / vtx.
// Chunks a handle's heavy-triangle list holds (4M (triangle, bin) pairs).
constexpr unsigned HEAVY_LIST_CAP = 16384;

// heavy (optional, heavy_cap entries): triangles spanning many bins are
// listed there in chunks of pairs, whose entries launch_scatter writes
// spread over whole CTAs; heavy_epoch
// must change between consecutive count passes of a handle (its parity
// picks the list's counter; the pass clears the other one).
void launch_setup_count(const RasterGeom& g, int T, const int* tris, int V, const int4* vtx,
                        BinRect* rect, unsigned* bin_count, DevStatus* st, int stats, int num_sms, cudaStream_t s,
                        const int4* clip_tris = nullptr, unsigned clip_cap = 0, int exact = 0,
                        uint2* heavy = nullptr, unsigned heavy_cap = 0, unsigned heavy_epoch = 0);
// Count pass and scan in one launch for a frame of at most one scan chunk of
// bins (scan_chunks(nbins) == 1): the count pass's last CTA scans.  Returns
// false (nothing launched) for larger frames, which take launch_setup_count
// and launch_scan.
bool launch_count_and_scan(const RasterGeom& g, int T, const int* tris, int V, const int4* vtx, BinRect* rect,
                           unsigned* bin_count, DevStatus* st, int stats, int num_sms, cudaStream_t s,
                           const int4* clip_tris, unsigned clip_cap, int exact, uint2* heavy, unsigned heavy_cap,
                           unsigned heavy_epoch, unsigned* bin_off, unsigned* cursor, unsigned long long capacity,
                           unsigned long long* chunk_state, unsigned scan_epoch);
// Near/far clipping of the triangles with a rejected vertex: sub-triangles
// (3 snapped points each) and their triangle's index appended at
// st->clip_count (PIKO_ERR_OVERFLOW past cap).
void launch_clip(int W, int H, int T, const int* tris, int V, const float* pos, const float* mvp, const int4* vtx,
                 int4* clip_tris, unsigned* clip_orig, unsigned cap, DevStatus* st, int num_sms, cudaStream_t s);
// chunk_state: scan_chunks(nbins) words, zero at allocation; epoch must
// differ between consecutive scans on the same state array.  wait_budget:
// clock cycles a look-back wait may take before PIKO_ERR_TIMEOUT; withhold:
// test hook bits (piko_scan.cuh).
void launch_scan(int nbins, unsigned* bin_count, unsigned* bin_off, unsigned* cursor, unsigned long long capacity,
                 DevStatus* st, unsigned long long* chunk_state, unsigned epoch, cudaStream_t s,
                 long long wait_budget = 40000000, int withhold = 0);
int scan_chunks(int nbins);
void launch_scatter(const RasterGeom& g, int T, const BinRect* rect, const unsigned* bin_off, unsigned* cursor,
                    unsigned* bin_tris, unsigned long long capacity, DevStatus* st, int num_sms, cudaStream_t s,
                    const int4* clip_tris = nullptr, unsigned clip_cap = 0, const int* tris = nullptr, int V = 0,
                    const int4* vtx = nullptr, const uint2* heavy = nullptr, unsigned heavy_cap = 0,
                    unsigned heavy_epoch = 0);
cudaError_t launch_process(const ProcessParams& p, int threads, int grid, cudaStream_t s);
cudaError_t process_occupancy(const ProcessParams& p, int threads, int* blocks_per_sm);

// Boxes (pixels of a triangle's bounding box inside a tile) up to this size
// take the warp's flattened walk when the triangle is below 128 pixels a
// side; larger boxes, and larger triangles, a whole warp per triangle.
constexpr int DEFAULT_SMALL_PX = 4096;

// Default CTA size of the Process stage for a tile of bin_px pixels in a
// frame of nbins tiles on num_sms SMs.  A frame with fewer tiles than twice
// the SMs (one CTA per tile cannot fill the GPU) takes 512 threads, so that
// a tile's queued large triangles spread over 16 warps instead of 4.
inline int default_process_threads(int bin_px, int nbins, int num_sms) {
  if (nbins < 2 * num_sms) return 512;
  return bin_px <= 64 ? 64 : (bin_px <= 256 ? 128 : 256);
}

// The two other pipeline mappings (piko_altpipe.cu): the fused one without
// tiling and the unfused five-stage one.  Stages run in this order:
// fused: ALT_RASTER_MIN, ALT_SHADE_PIXELS; unfused: ALT_RASTER_EMIT,
// ALT_FRAG_SHADE, ALT_FRAG_DEPTH, ALT_FRAG_COMPOSITE, ALT_CLEAR_EMPTY; the
// key buffer is set to all ones before the rasterizer.
enum { ALT_RASTER_MIN = 0, ALT_RASTER_EMIT, ALT_SHADE_PIXELS, ALT_FRAG_SHADE, ALT_FRAG_DEPTH, ALT_FRAG_COMPOSITE,
       ALT_CLEAR_EMPTY };
struct AltInputs {
  int W, H, T, V, mode, unclamped;
  const int* tris;
  const int4* vtx;
  const float* color;
  const float* normal;
  const float* light;
  const float* invw;
  unsigned long long* key;
  float4* rgba;
  uint2* gnorm;
  uint2* galb;
  DevStatus* st;
  const float* pos;                // positions and matrix (clipped winners' shading)
  const float* mvp;
  const int4* clip_tris;           // near/far clipping: sub-triangles (NULL: off)
  const unsigned* clip_orig;
  unsigned clip_cap;
  unsigned* frag_pix;              // fragment buffers (unfused): pixel, key, colour
  unsigned long long* frag_key;    //   (G-buffer mode: the colour slots hold the
  float4* frag_rgba;               //   normal and albedo halves)
  unsigned long long frag_cap;
};
cudaError_t alt_stage(const AltInputs& in, int stage, bool persp, int num_sms, cudaStream_t s);

void launch_deferred_light(int W, int H, const unsigned long long* key, const uint2* gnorm,
                           const uint2* galb, const float4* lights, int n_lights, float4* rgba,
                           int num_sms, cudaStream_t s);

}  // namespace piko
