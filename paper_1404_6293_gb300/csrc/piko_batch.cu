// piko_batch.cu -- many scenes in one pass.
//
// All scenes of a batch share one index space per phase: vertices,
// triangles, bins and tiles of scene s follow those of scenes 0..s-1, and a
// work item finds its scene by binary search over the prefix counts.  The
// phases are those of the single-scene forward (vertex stage, setup and
// counts, scan, scatter, Process); by default they run in one persistent
// cooperative launch whose CTAs meet at grid barriers between phases.  The
// Piko paper's runtime is multi-kernel and names a persistent kernel as the
// alternative it did not take (Sec. 5); the per-scene bin size and schedule
// are the knobs its Sec. 7.2 explores by hand.
//
// Every wait (grid barrier, scan look-back) is bounded by a clock budget;
// on expiry PIKO_ERR_TIMEOUT is recorded and every later phase is skipped.
#include <cstring>
#include <string>
#include <vector>

#include "piko_scan.cuh"
#include "piko_tile.cuh"
#include "piko_bwd_tile.cuh"

namespace piko {

struct BatchScene {
  RasterGeom g;
  int V, T, mode, schedule;
  int vtx_base, tri_base, bin_base, pix_base;
  int slot_bits, nslots, rec_stride;
  int unclamped;  // Lambert without the clamp (the handle's option)
  const float4* pos;
  const int* tris;
  const float* mvp;
  const float* color;
  const float* normal;
  const float* light;
  unsigned long long* key_out;
  float4* rgba_out;
  uint2* gnorm_out;
  uint2* galb_out;
  // backward
  const float4* dl;
  float* dcolor;
  float* dnormal;
  float* dlight;
};

struct BatchSync {
  unsigned count;     // CTAs arrived at the current grid barrier
  unsigned gen;       // barrier generation
  unsigned dyn_head;  // dynamic tile queue
  unsigned pad;
};

enum : int { PH_VERTEX = 1, PH_COUNT = 2, PH_SCAN = 4, PH_SCATTER = 8, PH_PROCESS = 16 };

struct BatchParams {
  int n;
  const BatchScene* sc;    // [n]
  const int* vtx_prefix;   // [n+1] each
  const int* tri_prefix;
  const int* bin_prefix;
  const int* stat_prefix;  // tiles of static scenes
  const int* dyn_prefix;   // tiles of dynamic scenes
  const int* btile_prefix;  // backward tiles (BWD_TILE_W x BATCH_BWD_TILE_H)
  int total_v, total_t, total_bins, total_static, total_dyn, total_btiles;
  int4* vtx;
  float* vdot;
  float* invw;  // 1 / clip w per vertex (perspective-correct attributes), else NULL
  BinRect* rect;
  unsigned* cnt;  // 2 * total_bins, zero between frames
  unsigned* bin_off;
  unsigned* cursor;
  unsigned long long* chunk_state;
  unsigned epoch;
  unsigned* bin_tris;
  unsigned long long capacity;
  DevStatus* st;
  BatchSync* sync;
  int phases;      // PH_* to run in this launch
  int persistent;  // grid barriers between phases
  int max_bin_px;
  long long wait_budget;  // clock cycles a device-side wait may take before PIKO_ERR_TIMEOUT
  int withhold;           // test hooks: TEST_WITHHOLD_* bits (piko_scan.cuh)
};

// largest s with prefix[s] <= i (prefix[n] > i)
__device__ __forceinline__ int find_scene(const int* __restrict__ prefix, int n, int i) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool skip_flags(const DevStatus* st) {
  return (*reinterpret_cast<const volatile unsigned*>(&st->flags) & STATUS_SKIP_MASK) != 0u;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier of a co-resident grid.  Returns false (for every thread of
// the CTA) when the frame must stop: a wait ran out of its budget or an
// earlier phase recorded a condition that makes later phases unsafe.
// skip_arrival (a test hook) makes this CTA wait without arriving, so that
// every CTA's wait runs out.
__device__ bool grid_barrier(BatchSync* sync, DevStatus* st, long long budget, bool skip_arrival = false) {
  __shared__ int s_go;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire_u32(&sync->gen);
    __threadfence();
    if (!skip_arrival && atomicAdd(&sync->count, 1u) == gridDim.x - 1) {
      sync->count = 0u;
      __threadfence();
      st_release_u32(&sync->gen, gen + 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_u32(&sync->gen) == gen) {
        if (clock64() - t0 > budget) {
          record_error(st, PIKO_ERR_TIMEOUT);
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    s_go = skip_flags(st) ? 0 : 1;  // one read per CTA: every thread takes the same branch
  }
  __syncthreads();
  return s_go != 0;
}

// The same stop test outside a barrier, uniform over the CTA.
__device__ bool cta_should_stop(const DevStatus* st) {
  __shared__ int s_stop;
  __syncthreads();
  if (threadIdx.x == 0) s_stop = skip_flags(st) ? 1 : 0;
  __syncthreads();
  return s_stop != 0;
}

// ------------------------------------------------------------------ phases
template <bool PERSP>
__device__ void phase_vertex(const BatchParams& b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.total_v; i += gridDim.x * blockDim.x) {
    const int s = find_scene(b.vtx_prefix, b.n, i);
    const BatchScene& d = b.sc[s];
    const int v = i - d.vtx_base;
    if (PERSP) {
      float w;
      b.vtx[i] = snap_vertex(__ldg(d.pos + v), d.mvp, (float)d.g.W, (float)d.g.H, &w);
      b.invw[i] = w > 0.0f ? __fdiv_rn(1.0f, w) : 0.0f;
    } else {
      b.vtx[i] = snap_vertex(__ldg(d.pos + v), d.mvp, (float)d.g.W, (float)d.g.H);
    }
    if (d.mode == PIKO_SHADE_LAMBERT) {
      const float* n = d.normal + 3 * (size_t)v;
      b.vdot[i] = __ldg(n) * __ldg(d.light) + __ldg(n + 1) * __ldg(d.light + 1) + __ldg(n + 2) * __ldg(d.light + 2);
    }
  }
}

struct LaneBins {
  bool valid, single;
  int bx0, by0, bx1, by1;
  int nbx, bin_base;
};

__device__ __forceinline__ LaneBins lane_setup(const BatchParams& b, int t) {
  LaneBins r;
  r.valid = false; r.single = false;
  r.bx0 = 0; r.by0 = 0; r.bx1 = -1; r.by1 = -1; r.nbx = 1; r.bin_base = 0;
  if (t >= b.total_t) return r;
  const int s = find_scene(b.tri_prefix, b.n, t);
  const BatchScene& d = b.sc[s];
  r.nbx = d.g.nbx;
  r.bin_base = d.bin_base;
  const int tl = t - d.tri_base;
  const int ia = __ldg(d.tris + 3 * (size_t)tl), ib = __ldg(d.tris + 3 * (size_t)tl + 1),
            ic = __ldg(d.tris + 3 * (size_t)tl + 2);
  if ((unsigned)ia >= (unsigned)d.V || (unsigned)ib >= (unsigned)d.V || (unsigned)ic >= (unsigned)d.V) {
    record_error(b.st, PIKO_ERR_BAD_INDEX);
    return r;
  }
  const int4* vtx = b.vtx + d.vtx_base;
  const int4 p0 = __ldg(vtx + ia), p1 = __ldg(vtx + ib), p2 = __ldg(vtx + ic);
  if (!(p0.w & p1.w & p2.w)) return r;
  const long long A = (long long)(p1.x - p0.x) * (p2.y - p0.y) - (long long)(p2.x - p0.x) * (p1.y - p0.y);
  if (A == 0) return r;
  int px0, px1, py0, py1;
  centre_range(min(p0.x, min(p1.x, p2.x)), max(p0.x, max(p1.x, p2.x)), 0, d.g.W - 1, px0, px1);
  centre_range(min(p0.y, min(p1.y, p2.y)), max(p0.y, max(p1.y, p2.y)), 0, d.g.H - 1, py0, py1);
  if (px0 > px1 || py0 > py1) return r;
  r.valid = true;
  r.bx0 = px0 >> d.g.bshift_x; r.bx1 = px1 >> d.g.bshift_x;
  r.by0 = py0 >> d.g.bshift_y; r.by1 = py1 >> d.g.bshift_y;
  r.single = r.bx0 == r.bx1 && r.by0 == r.by1;
  return r;
}

// Pairs (triangle, bin) of multi-bin triangles, spread over the warp.
template <typename F>
__device__ __forceinline__ void for_multi_pairs(const LaneBins& r, int lane, F&& f) {
  const int bw = r.bx1 - r.bx0 + 1;
  const int nb = (r.valid && !r.single) ? bw * (r.by1 - r.by0 + 1) : 0;
  int incl = nb;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(FULL_MASK, incl, o);
    if (lane >= o) incl += u;
  }
  const int total = __shfl_sync(FULL_MASK, incl, 31);
  for (int k0 = 0; k0 < total; k0 += 32) {
    const int k = k0 + lane;
    const int kk = k < total ? k : total - 1;
    int owner = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      const int v = __shfl_sync(FULL_MASK, incl, owner + s - 1);
      if (v <= kk) owner += s;
    }
    const int ox = __shfl_sync(FULL_MASK, r.bx0, owner), oy = __shfl_sync(FULL_MASK, r.by0, owner);
    const int obw = __shfl_sync(FULL_MASK, bw, owner);
    const int first = __shfl_sync(FULL_MASK, incl - nb, owner);
    const int onbx = __shfl_sync(FULL_MASK, r.nbx, owner), obase = __shfl_sync(FULL_MASK, r.bin_base, owner);
    if (k < total) {
      const int local = k - first;
      const int yy = local / obw;
      f(owner, obase + (oy + yy) * onbx + ox + (local - yy * obw));
    }
  }
}

__device__ void phase_count(const BatchParams& b) {
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < b.total_t;
       base += warps_total * 32) {
    const int t = base + lane;
    const LaneBins r = lane_setup(b, t);
    const unsigned bin = r.single ? (unsigned)(r.bin_base + r.by0 * r.nbx + r.bx0) : 0xFFFFFFFFu;
    const unsigned grp = __match_any_sync(FULL_MASK, bin);
    const int leader = __ffs(grp) - 1;
    unsigned slot = 0;
    if (r.single && lane == leader) slot = atomicAdd(b.cnt + bin, (unsigned)__popc(grp));
    slot = __shfl_sync(FULL_MASK, slot, leader) + __popc(grp & lt_mask);
    if (t < b.total_t) {
      BinRect q;
      if (!r.valid) {
        q.lo = 0xFFFFFFFFu; q.hi = 0u;
      } else if (r.single) {
        q.lo = (unsigned)r.bx0 | ((unsigned)r.by0 << 16) | 0x8000u; q.hi = slot;
      } else {
        q.lo = (unsigned)r.bx0 | ((unsigned)r.by0 << 16); q.hi = (unsigned)r.bx1 | ((unsigned)r.by1 << 16);
      }
      b.rect[t] = q;
    }
    for_multi_pairs(r, lane, [&](int, int gbin) { atomicAdd(b.cnt + b.total_bins + gbin, 1u); });
  }
}

__device__ void phase_scan(const BatchParams& b, ScanSmem& sm) {
  const int chunk_bins = (int)blockDim.x * SCAN_PER;
  const int nchunks = (b.total_bins + chunk_bins - 1) / chunk_bins;
  // tickets only grow, so a CTA takes at most nchunks + 1 of them; the cap
  // turns a broken ticket counter into a recorded error instead of a spin
  for (int iter = 0;; ++iter) {
    if (threadIdx.x == 0) {
      sm.chunk = (int)atomicAdd(&b.st->scan_ticket, 1u);
      if (iter > nchunks) {
        record_error(b.st, PIKO_ERR_TIMEOUT);
        sm.chunk = nchunks;
      }
    }
    __syncthreads();
    const int chunk = sm.chunk;
    if (chunk < 0 || chunk >= nchunks) break;
    scan_chunk(chunk, nchunks, b.total_bins, b.cnt, b.bin_off, b.cursor, b.capacity, b.st, b.chunk_state, b.epoch,
               sm, &b.sync->dyn_head, b.wait_budget, b.withhold);
    __syncthreads();  // sm.chunk is rewritten for the next ticket
  }
}

__device__ void phase_scatter(const BatchParams& b) {
  const int lane = threadIdx.x & 31;
  const int warps_total = gridDim.x * (blockDim.x >> 5);
  for (int base = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < b.total_t;
       base += warps_total * 32) {
    const int t = base + lane;
    LaneBins r;
    r.valid = false; r.single = false;
    r.bx0 = 0; r.by0 = 0; r.bx1 = -1; r.by1 = -1; r.nbx = 1; r.bin_base = 0;
    if (t < b.total_t) {
      const BinRect q = b.rect[t];
      if (q.lo != 0xFFFFFFFFu) {
        const BatchScene& d = b.sc[find_scene(b.tri_prefix, b.n, t)];
        r.valid = true;
        r.nbx = d.g.nbx;
        r.bin_base = d.bin_base;
        if (q.lo & 0x8000u) {
          r.single = true;
          const int gbin = d.bin_base + (int)(q.lo >> 16) * d.g.nbx + (int)(q.lo & 0x7FFFu);
          const unsigned pos = __ldg(b.bin_off + gbin) + q.hi;
          if (pos < b.capacity) b.bin_tris[pos] = (unsigned)t;
        } else {
          r.bx0 = q.lo & 0xFFFF; r.by0 = q.lo >> 16; r.bx1 = q.hi & 0xFFFF; r.by1 = q.hi >> 16;
        }
      }
    }
    for_multi_pairs(r, lane, [&](int owner, int gbin) {
      const unsigned pos = atomicAdd(b.cursor + gbin, 1u);
      if (pos < b.capacity) b.bin_tris[pos] = (unsigned)(base + owner);
    });
  }
}

struct ProcessShared {
  TileScene sc;
  int tile, scene;
  unsigned nbig;
};

__device__ void load_tile_scene(const BatchParams& b, int s, TileScene& t) {
  const BatchScene& d = b.sc[s];
  t.g = d.g;
  t.mode = d.mode;
  t.unclamped = d.unclamped;
  t.small_px = 32;
  t.slot_bits = d.slot_bits;
  t.nslots = d.nslots;
  t.rec_stride = d.rec_stride;
  t.tri_base = d.tri_base;
  t.tris = d.tris;
  t.vtx = b.vtx + d.vtx_base;
  t.color = d.color;
  t.normal = d.normal;
  t.light = d.light;
  t.vdot = b.vdot + d.vtx_base;
  t.invw = b.invw ? b.invw + d.vtx_base : nullptr;
  t.T = d.T;
  t.clip_tris = nullptr;  // batches do not clip
  t.clip_orig = nullptr;
  t.pos = nullptr;
  t.mvp = nullptr;
  t.key_out = d.key_out;
  t.rgba_out = d.rgba_out;
  t.gnorm_out = d.gnorm_out;
  t.galb_out = d.galb_out;
}

template <bool PERSP>
__device__ void process_one(const BatchParams& b, const int* prefix, int i, ProcessShared& ps, const TileSmem& sm,
                            unsigned& big_base) {
  if (threadIdx.x == 0) {
    const int s = find_scene(prefix, b.n, i);
    if (s != ps.scene) {
      load_tile_scene(b, s, ps.sc);
      ps.scene = s;
    }
    ps.tile = i - __ldg(prefix + s);
  }
  __syncthreads();
  const TileScene& sc = ps.sc;
  const int gbin = b.sc[ps.scene].bin_base + ps.tile;
  TileStats st = {0ull, 0ull, 0ull};
  const unsigned beg = __ldg(b.bin_off + gbin), end = __ldg(b.bin_off + gbin + 1);
  if (beg > end || (unsigned long long)end > b.capacity) {  // same for every thread: skip the tile
    if (threadIdx.x == 0) record_error(b.st, PIKO_ERR_OVERFLOW);
    __syncthreads();
    return;
  }
  process_tile<false, PERSP>(sc, ps.tile, beg, end, b.bin_tris, sm, big_base, st);
}

template <bool PERSP>
__device__ void phase_process(const BatchParams& b, ProcessShared& ps, const TileSmem& sm) {
  for (int i = threadIdx.x; i < b.max_bin_px; i += blockDim.x) sm.skey[i] = KEY_EMPTY;
  if (threadIdx.x == 0) {
    ps.scene = -1;
    *sm.s_nbig = 0u;
  }
  __syncthreads();
  unsigned big_base = 0u;
  // DirectMap scenes: tiles dealt round robin; then LoadBalance scenes from the queue
  for (int i = blockIdx.x; i < b.total_static; i += gridDim.x) process_one<PERSP>(b, b.stat_prefix, i, ps, sm, big_base);
  __shared__ int s_next;
  for (int iter = 0;; ++iter) {
    if (threadIdx.x == 0) {
      s_next = (int)atomicAdd(&b.sync->dyn_head, 1u);
      if (iter > b.total_dyn) {  // the queue only grows: at most total_dyn + 1 takes
        record_error(b.st, PIKO_ERR_TIMEOUT);
        s_next = b.total_dyn;
      }
    }
    __syncthreads();
    const int i = s_next;
    __syncthreads();  // s_next is rewritten for the next tile
    if (i < 0 || i >= b.total_dyn) break;
    process_one<PERSP>(b, b.dyn_prefix, i, ps, sm, big_base);
  }
}

#ifndef PIKO_BATCH_MAXNREG
#define PIKO_BATCH_MAXNREG 64
#endif
#ifndef PIKO_BATCH_THREADS
#define PIKO_BATCH_THREADS 128
#endif
constexpr int BATCH_THREADS = PIKO_BATCH_THREADS;  // CTA size of the persistent batch kernel

// PERSP: perspective-correct attributes; one instance per setting
template <bool PERSP>
__global__ void __maxnreg__(PIKO_BATCH_MAXNREG) k_batch_forward(BatchParams b) {
  extern __shared__ __align__(16) unsigned long long smem[];
  __shared__ ScanSmem scan_sm;
  __shared__ ProcessShared ps;
  __shared__ unsigned s_nbig;
  TileSmem sm;
  sm.skey = smem;
  sm.sbig = reinterpret_cast<int*>(smem + b.max_bin_px);
  sm.sfrag = sm.sbig + blockDim.x;
  sm.srec = sm.sfrag + (blockDim.x >> 5) * FRAG_WARP_WORDS;
  sm.s_nbig = &s_nbig;
  if (cta_should_stop(b.st)) return;
  if (b.phases & PH_VERTEX) {
    phase_vertex<PERSP>(b);
    const bool skip = (b.withhold & TEST_WITHHOLD_BARRIER) && blockIdx.x == 0;
    if (b.persistent && !grid_barrier(b.sync, b.st, b.wait_budget, skip)) return;
  }
  if (b.phases & PH_COUNT) {
    if (blockIdx.x == 0 && threadIdx.x == 0) b.st->scan_ticket = 0u;  // the scan runs after a barrier
    phase_count(b);
    if (b.persistent && !grid_barrier(b.sync, b.st, b.wait_budget)) return;
  }
  if (b.phases & PH_SCAN) {
    phase_scan(b, scan_sm);
    if (b.persistent && !grid_barrier(b.sync, b.st, b.wait_budget)) return;
  }
  if (b.phases & PH_SCATTER) {
    if (cta_should_stop(b.st)) return;
    phase_scatter(b);
    if (b.persistent && !grid_barrier(b.sync, b.st, b.wait_budget)) return;
  }
  if (b.phases & PH_PROCESS) {
    if (cta_should_stop(b.st)) return;
    phase_process<PERSP>(b, ps, sm);
  }
}

// ------------------------------------------------------------------ backward
// BWD_TILE_W x BATCH_BWD_TILE_H tiles of every scene, dealt round robin; each tile's gradients are
// accumulated as in the single-scene backward.
struct BatchBwdParams {
  int n;
  const BatchScene* sc;
  const int* btile_prefix;  // [n+1] backward tiles per scene
  int total_btiles;
  const int4* vtx;
  const float* invw;  // as in BatchParams
};

// Warp form: each warp takes whole tiles (grid-stride over the batch's
// tiles), with no CTA barrier; the scene of a tile is found by every lane
// (uniform loads) and its descriptor kept in the warp's shared slot (in
// registers it would cost the tile loop its occupancy).
constexpr int BATCH_BWD_WARPS = BWD_THREADS / 32;
struct BatchBwdSmem {
  float stage[BATCH_BWD_WARPS][BWD_VALS][33];
  BwdScene sc[BATCH_BWD_WARPS];
};
template <bool PERSP>
#ifndef PIKO_BWD_MINB
#define PIKO_BWD_MINB 3
#endif
__global__ void __launch_bounds__(BWD_THREADS, PIKO_BWD_MINB) k_batch_backward(BatchBwdParams b) {
  extern __shared__ __align__(16) unsigned char bwd_smem_raw[];
  BatchBwdSmem& sm = *reinterpret_cast<BatchBwdSmem*>(bwd_smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * BATCH_BWD_WARPS;
  BwdScene& c = sm.sc[warp];
  for (int i = blockIdx.x * BATCH_BWD_WARPS + warp; i < b.total_btiles; i += nwarps) {
    const int s = find_scene(b.btile_prefix, b.n, i);
    const BatchScene& d = b.sc[s];
    if (d.dl == nullptr || d.mode == PIKO_SHADE_GBUFFER) continue;  // the same for the whole warp
    __syncwarp();  // the previous tile's reads of c are done
    if (lane == 0) {
      c.W = d.g.W; c.H = d.g.H; c.mode = d.mode; c.unclamped = d.unclamped; c.T = d.T; c.V = d.V;
      c.tris = d.tris; c.vtx = b.vtx + d.vtx_base; c.color = d.color; c.normal = d.normal; c.light = d.light;
      c.invw = b.invw ? b.invw + d.vtx_base : nullptr;
      c.pos = nullptr;  // batches do not clip
      c.mvp = nullptr;
      c.key = d.key_out; c.dl = d.dl; c.dcolor = d.dcolor; c.dnormal = d.dnormal; c.dlight = d.dlight;
    }
    __syncwarp();
    float L0 = 0.f, L1 = 0.f, L2 = 0.f;
    if (c.mode == PIKO_SHADE_LAMBERT) {
      L0 = __ldg(c.light); L1 = __ldg(c.light + 1); L2 = __ldg(c.light + 2);
    }
    const int lt = i - __ldg(b.btile_prefix + s);
    const int ntx = (c.W + BWD_TILE_W - 1) / BWD_TILE_W;
    const int ty = lt / ntx, tx = lt - ty * ntx;
    backward_warp_tile<PERSP, false, BATCH_BWD_TILE_H>(c, tx * BWD_TILE_W, ty * BATCH_BWD_TILE_H, sm.stage[warp],
                                                        L0, L1, L2);
  }
}
constexpr size_t BATCH_BWD_SMEM = sizeof(BatchBwdSmem);

}  // namespace piko

// =====================================================================
// Host side: layout, scratch, launches (called from the C ABI in piko_api.cu)
// =====================================================================

using namespace piko;

namespace {

int ilog2i(int v) {
  int s = 0;
  while ((1 << s) < v) ++s;
  return s;
}

}  // namespace

// Everything the batch keeps between calls; owned by the handle.
struct BatchState {
  // device scratch
  void* desc = nullptr;  // scenes + prefix arrays
  size_t desc_cap = 0;
  int4* vtx = nullptr;
  long long vcap = 0;
  float* vdot = nullptr;
  long long dcap = 0;
  float* invw = nullptr;
  long long icap = 0;
  BinRect* rect = nullptr;
  long long tcap = 0;
  unsigned* cnt = nullptr;
  unsigned* bin_off = nullptr;
  unsigned* cursor = nullptr;
  unsigned long long* chunk_state = nullptr;
  long long bcap = 0;  // bins
  unsigned* bin_tris = nullptr;
  long long ecap = 0;
  BatchSync* sync = nullptr;
  unsigned epoch = 0;
  // host staging (pinned) and the last layout
  void* staging = nullptr;
  size_t staging_cap = 0;
  cudaEvent_t uploaded = nullptr;
  BatchParams params;
  std::vector<BatchScene> host_desc;  // the uploaded descriptors
  size_t smem = 0;
  int grid = 0;
  int n = 0;
  int persp = 0;               // the layout's attribute interpolation (perspective-correct or not)
  long long last_entries = 0;  // bin entries of the last frame read back (sizes the shading records)
  long long last_bins = 0;     // bins of that frame
};

namespace {

template <typename T>
int grow_dev(T** p, long long* cap, long long need, bool zero, std::string& err) {
  if (need <= *cap) return PIKO_OK;
  const long long n = need + need / 4 + 1024;
  if (*p) {
    if (cudaDeviceSynchronize() != cudaSuccess) { err = "synchronize before growing batch scratch"; return PIKO_ERR_CUDA; }
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
  }
  if (cudaMalloc(reinterpret_cast<void**>(p), (size_t)n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    err = "cudaMalloc of batch scratch failed";
    return PIKO_ERR_OOM;
  }
  if (zero && cudaMemset(*p, 0, (size_t)n * sizeof(T)) != cudaSuccess) {
    err = "cudaMemset of batch scratch failed";
    return PIKO_ERR_CUDA;
  }
  *cap = n;
  return PIKO_OK;
}

bool valid_bin(int b) { return b == 8 || b == 16 || b == 32 || b == 64; }
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

void batch_state_free(BatchState* bs) {
  if (!bs) return;
  cudaFree(bs->desc);
  cudaFree(bs->vtx);
  cudaFree(bs->vdot);
  cudaFree(bs->invw);
  cudaFree(bs->rect);
  cudaFree(bs->cnt);
  cudaFree(bs->bin_off);
  cudaFree(bs->cursor);
  cudaFree(bs->chunk_state);
  cudaFree(bs->bin_tris);
  cudaFree(bs->sync);
  if (bs->staging) cudaFreeHost(bs->staging);
  if (bs->uploaded) cudaEventDestroy(bs->uploaded);
  cudaGetLastError();
  delete bs;
}

// Builds the descriptors, sizes the scratch and uploads the layout.
// Returns a PIKO_* code; err describes a failure.
int batch_prepare(BatchState*& bs, int num_sms, const piko_scene* scenes, int n, piko_framebuffer* fbs,
                  const int32_t* bin_sizes, const int32_t* schedules, int default_bin_w, int default_bin_h,
                  int default_schedule, int unclamped, int persp, cudaStream_t stream, std::string& err) {
  if (!bs) bs = new BatchState();
  if (n < 1 || !scenes || !fbs) { err = "batch needs n >= 1 scenes and framebuffers"; return PIKO_ERR_INVALID_ARG; }
  std::vector<BatchScene> d(n);
  std::vector<int> pv(n + 1), pt(n + 1), pb(n + 1), ps(n + 1), pd(n + 1), pp(n + 1);
  long long tv = 0, tt = 0, tb = 0, tsd = 0, tdy = 0, tp = 0;
  int max_bin_px = 64, max_rec = 0;
  // shading records per tile from the last frame's mean entries per bin
  const int slots_hint = bs ? slots_for_entries(bs->last_entries, (int)(bs->last_bins > 0 ? bs->last_bins : 1)) : 0;
  for (int i = 0; i < n; ++i) {
    const piko_scene& s = scenes[i];
    const piko_framebuffer& f = fbs[i];
    const int bw = bin_sizes ? bin_sizes[2 * i] : default_bin_w, bh = bin_sizes ? bin_sizes[2 * i + 1] : default_bin_h;
    int sched = schedules ? schedules[i] : default_schedule;
    if (s.width < 1 || s.height < 1 || s.width > 32767 || s.height > 32767 || !valid_bin(bw) || !valid_bin(bh) ||
        s.num_vertices < 0 || s.num_triangles < 0 || s.reserved != 0 || sched < PIKO_SCHED_STATIC ||
        sched > PIKO_SCHED_HARDWARE || s.shade_mode < PIKO_SHADE_GOURAUD || s.shade_mode > PIKO_SHADE_GBUFFER ||
        !f.key || (s.num_vertices > 0 && (!s.pos || !aligned16(s.pos))) || (s.num_triangles > 0 && !s.tris) ||
        (s.num_triangles > 0 && s.shade_mode == PIKO_SHADE_GOURAUD && !s.color) ||
        (s.num_triangles > 0 && s.shade_mode != PIKO_SHADE_GOURAUD && !s.normal) ||
        (s.shade_mode == PIKO_SHADE_LAMBERT && !s.light_dir) ||
        (s.shade_mode == PIKO_SHADE_GBUFFER && (!f.gbuf_normal || !f.gbuf_albedo))) {
      err = "invalid scene " + std::to_string(i) + " in batch";
      return PIKO_ERR_INVALID_ARG;
    }
    if (sched == PIKO_SCHED_HARDWARE) sched = PIKO_SCHED_DYNAMIC;
    BatchScene& x = d[i];
    std::memset(&x, 0, sizeof(x));
    x.g.W = s.width; x.g.H = s.height;
    x.g.bshift_x = ilog2i(bw); x.g.bshift_y = ilog2i(bh);
    x.g.nbx = (s.width + bw - 1) / bw; x.g.nby = (s.height + bh - 1) / bh;
    x.V = s.num_vertices; x.T = s.num_triangles; x.mode = s.shade_mode; x.schedule = sched;
    x.vtx_base = (int)tv; x.tri_base = (int)tt; x.bin_base = (int)tb; x.pix_base = 0;
    tile_layout(s.num_triangles, bw * bh, s.shade_mode, s.color != nullptr, persp != 0, 255, x.slot_bits, x.nslots,
                x.rec_stride, slots_hint);
    x.unclamped = unclamped;
    x.pos = reinterpret_cast<const float4*>(s.pos);
    x.tris = s.tris; x.mvp = s.mvp; x.color = s.color; x.normal = s.normal; x.light = s.light_dir;
    x.key_out = reinterpret_cast<unsigned long long*>(f.key);
    x.rgba_out = reinterpret_cast<float4*>(f.rgba);
    x.gnorm_out = reinterpret_cast<uint2*>(f.gbuf_normal);
    x.galb_out = reinterpret_cast<uint2*>(f.gbuf_albedo);
    const int ntiles = x.g.nbx * x.g.nby;
    pv[i] = (int)tv; pt[i] = (int)tt; pb[i] = (int)tb; ps[i] = (int)tsd; pd[i] = (int)tdy; pp[i] = (int)tp;
    tv += x.V; tt += x.T; tb += ntiles;
    tp += (long long)((s.width + BWD_TILE_W - 1) / BWD_TILE_W) *
          ((s.height + BATCH_BWD_TILE_H - 1) / BATCH_BWD_TILE_H);
    if (sched == PIKO_SCHED_STATIC) tsd += ntiles;
    else tdy += ntiles;
    if (bw * bh > max_bin_px) max_bin_px = bw * bh;
    if (x.nslots * x.rec_stride > max_rec) max_rec = x.nslots * x.rec_stride;
  }
  pv[n] = (int)tv; pt[n] = (int)tt; pb[n] = (int)tb; ps[n] = (int)tsd; pd[n] = (int)tdy; pp[n] = (int)tp;
  if (tv >= (1LL << 31) || tt >= (1LL << 31) || tb >= (1LL << 31) || tp >= (1LL << 31)) {
    err = "batch too large (a total reaches 2^31)";
    return PIKO_ERR_INVALID_ARG;
  }
  // device scratch
  int r;
  if ((r = grow_dev(&bs->vtx, &bs->vcap, tv, false, err)) != PIKO_OK) return r;
  if ((r = grow_dev(&bs->vdot, &bs->dcap, tv, false, err)) != PIKO_OK) return r;
  if (persp && (r = grow_dev(&bs->invw, &bs->icap, tv, false, err)) != PIKO_OK) return r;
  if ((r = grow_dev(&bs->rect, &bs->tcap, tt, false, err)) != PIKO_OK) return r;
  if (tb > bs->bcap) {
    // counts must start at zero; offsets/cursors/chunk states are rewritten
    cudaFree(bs->cnt); cudaFree(bs->bin_off); cudaFree(bs->cursor); cudaFree(bs->chunk_state);
    bs->cnt = nullptr; bs->bin_off = nullptr; bs->cursor = nullptr; bs->chunk_state = nullptr;
    const long long cap = tb + tb / 4 + 1024;
    const long long chunks = cap / (BATCH_THREADS * SCAN_PER) + 2;
    if (cudaMalloc(&bs->cnt, sizeof(unsigned) * 2 * (size_t)cap) != cudaSuccess ||
        cudaMalloc(&bs->bin_off, sizeof(unsigned) * (size_t)(cap + 1)) != cudaSuccess ||
        cudaMalloc(&bs->cursor, sizeof(unsigned) * (size_t)cap) != cudaSuccess ||
        cudaMalloc(&bs->chunk_state, sizeof(unsigned long long) * (size_t)chunks) != cudaSuccess ||
        cudaMemset(bs->cnt, 0, sizeof(unsigned) * 2 * (size_t)cap) != cudaSuccess ||
        cudaMemset(bs->chunk_state, 0, sizeof(unsigned long long) * (size_t)chunks) != cudaSuccess) {
      cudaGetLastError();
      err = "cudaMalloc of batch bins failed";
      return PIKO_ERR_OOM;
    }
    bs->bcap = cap;
  }
  if (bs->ecap == 0 && (r = grow_dev(&bs->bin_tris, &bs->ecap, 2 * tt + 4096, false, err)) != PIKO_OK) return r;
  if (!bs->sync) {
    if (cudaMalloc(&bs->sync, sizeof(BatchSync)) != cudaSuccess || cudaMemset(bs->sync, 0, sizeof(BatchSync)) != cudaSuccess) {
      err = "cudaMalloc of batch barrier failed";
      return PIKO_ERR_OOM;
    }
  }
  // descriptors + 6 prefix arrays, uploaded from pinned memory
  const size_t dbytes = sizeof(BatchScene) * n;
  const size_t pbytes = sizeof(int) * (n + 1);
  const size_t total = dbytes + 6 * pbytes;
  if (!bs->uploaded && cudaEventCreateWithFlags(&bs->uploaded, cudaEventDisableTiming) != cudaSuccess) {
    err = "cudaEventCreate failed";
    return PIKO_ERR_CUDA;
  }
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(stream, &cap_status);
  if (cap_status == cudaStreamCaptureStatusNone && bs->staging) cudaEventSynchronize(bs->uploaded);
  if (total > bs->staging_cap) {
    if (cap_status != cudaStreamCaptureStatusNone) {
      err = "batch layout grew during stream capture: call once before capturing";
      return PIKO_ERR_INVALID_ARG;
    }
    if (bs->staging) cudaFreeHost(bs->staging);
    cudaFree(bs->desc);
    bs->staging = nullptr; bs->desc = nullptr; bs->staging_cap = 0;
    const size_t cap = total + total / 2 + 4096;
    if (cudaMallocHost(&bs->staging, cap) != cudaSuccess || cudaMalloc(&bs->desc, cap) != cudaSuccess) {
      err = "allocation of batch descriptors failed";
      return PIKO_ERR_OOM;
    }
    bs->staging_cap = cap;
    bs->desc_cap = cap;
  }
  char* h = static_cast<char*>(bs->staging);
  std::memcpy(h, d.data(), dbytes);
  const std::vector<int>* arrays[6] = {&pv, &pt, &pb, &ps, &pd, &pp};
  for (int a = 0; a < 6; ++a) std::memcpy(h + dbytes + a * pbytes, arrays[a]->data(), pbytes);
  if (cudaMemcpyAsync(bs->desc, bs->staging, total, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaEventRecord(bs->uploaded, stream) != cudaSuccess) {
    err = "upload of batch descriptors failed";
    return PIKO_ERR_CUDA;
  }
  char* dd = static_cast<char*>(bs->desc);
  BatchParams& b = bs->params;
  std::memset(&b, 0, sizeof(b));
  b.n = n;
  b.sc = reinterpret_cast<const BatchScene*>(dd);
  b.vtx_prefix = reinterpret_cast<const int*>(dd + dbytes);
  b.tri_prefix = reinterpret_cast<const int*>(dd + dbytes + pbytes);
  b.bin_prefix = reinterpret_cast<const int*>(dd + dbytes + 2 * pbytes);
  b.stat_prefix = reinterpret_cast<const int*>(dd + dbytes + 3 * pbytes);
  b.dyn_prefix = reinterpret_cast<const int*>(dd + dbytes + 4 * pbytes);
  b.btile_prefix = reinterpret_cast<const int*>(dd + dbytes + 5 * pbytes);
  b.total_v = (int)tv; b.total_t = (int)tt; b.total_bins = (int)tb; b.total_static = (int)tsd;
  b.total_dyn = (int)tdy; b.total_btiles = (int)tp;
  b.vtx = bs->vtx; b.vdot = bs->vdot; b.invw = persp ? bs->invw : nullptr; b.rect = bs->rect; b.cnt = bs->cnt; b.bin_off = bs->bin_off;
  b.cursor = bs->cursor; b.chunk_state = bs->chunk_state; b.bin_tris = bs->bin_tris;
  b.capacity = (unsigned long long)bs->ecap; b.sync = bs->sync;
  b.max_bin_px = max_bin_px;
  bs->smem = tile_smem_bytes(max_bin_px, BATCH_THREADS, 1, 0) + (size_t)max_rec * 4;
  const auto kf = persp ? k_batch_forward<true> : k_batch_forward<false>;
  if (bs->smem > 48 * 1024 &&
      cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs->smem) != cudaSuccess) {
    err = "batch shared memory request refused";
    return PIKO_ERR_CUDA;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, BATCH_THREADS, bs->smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    err = "batch kernel does not fit on an SM";
    return PIKO_ERR_CUDA;
  }
  bs->grid = per_sm * num_sms;
  bs->n = n;
  bs->persp = persp ? 1 : 0;
  bs->host_desc = d;
  return PIKO_OK;
}

// Launches the forward phases; persistent = one cooperative launch.
int batch_launch_forward(BatchState* bs, DevStatus* st, bool persistent, cudaStream_t stream, std::string& err,
                         long long wait_budget, int withhold) {
  BatchParams b = bs->params;
  b.st = st;
  b.wait_budget = wait_budget;
  b.withhold = withhold;
  b.capacity = (unsigned long long)bs->ecap;
  b.bin_tris = bs->bin_tris;
  b.epoch = ++bs->epoch;
  if (cudaMemsetAsync(bs->sync, 0, sizeof(BatchSync), stream) != cudaSuccess) {
    err = "batch barrier reset failed";
    return PIKO_ERR_CUDA;
  }
  if (persistent) {
    b.phases = PH_VERTEX | PH_COUNT | PH_SCAN | PH_SCATTER | PH_PROCESS;
    b.persistent = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(bs->grid);
    cfg.blockDim = dim3(BATCH_THREADS);
    cfg.dynamicSmemBytes = bs->smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeCooperative;
    attr.val.cooperative = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, bs->persp ? k_batch_forward<true> : k_batch_forward<false>, b);
    if (e != cudaSuccess) {
      err = std::string("cooperative batch launch: ") + cudaGetErrorString(e);
      return PIKO_ERR_CUDA;
    }
    return PIKO_OK;
  }
  b.persistent = 0;
  const int phases[5] = {PH_VERTEX, PH_COUNT, PH_SCAN, PH_SCATTER, PH_PROCESS};
  for (int k = 0; k < 5; ++k) {
    b.phases = phases[k];
    if (bs->persp)
      k_batch_forward<true><<<bs->grid, BATCH_THREADS, bs->smem, stream>>>(b);
    else
      k_batch_forward<false><<<bs->grid, BATCH_THREADS, bs->smem, stream>>>(b);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("batch launch: ") + cudaGetErrorString(e);
    return PIKO_ERR_CUDA;
  }
  return PIKO_OK;
}

long long batch_capacity(const BatchState* bs) { return bs ? bs->ecap : 0; }

void batch_note_entries(BatchState* bs, long long entries) {
  if (!bs) return;
  bs->last_entries = entries;
  bs->last_bins = bs->params.total_bins;
}

int batch_grow_entries(BatchState* bs, long long need, std::string& err) {
  return grow_dev(&bs->bin_tris, &bs->ecap, need, false, err);
}

int batch_launch_backward(BatchState* bs, const piko_scene* scenes, int n, const piko_framebuffer* fbs,
                          const float* const* dl, float* const* dc, float* const* dn, float* const* dlt, int num_sms,
                          cudaStream_t stream, std::string& err) {
  if (!bs || bs->n != n) {
    err = "backward_batch needs a forward_batch of the same scenes first";
    return PIKO_ERR_INVALID_ARG;
  }
  // per-scene gradient pointers go into the descriptors (same layout)
  std::vector<BatchScene> d = bs->host_desc;
  for (int i = 0; i < n; ++i) {
    if (scenes[i].num_triangles != d[i].T || scenes[i].num_vertices != d[i].V ||
        reinterpret_cast<unsigned long long*>(fbs[i].key) != d[i].key_out) {
      err = "backward_batch scenes differ from the last forward_batch";
      return PIKO_ERR_INVALID_ARG;
    }
    if (dl && dl[i] && !aligned16(dl[i])) {
      err = "dl_drgba must be 16-byte aligned";
      return PIKO_ERR_INVALID_ARG;
    }
    d[i].dl = dl ? reinterpret_cast<const float4*>(dl[i]) : nullptr;
    d[i].dcolor = dc ? dc[i] : nullptr;
    d[i].dnormal = dn ? dn[i] : nullptr;
    d[i].dlight = dlt ? dlt[i] : nullptr;
    d[i].color = scenes[i].color;
    d[i].normal = scenes[i].normal;
    d[i].light = scenes[i].light_dir;
  }
  cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(stream, &cap_status);
  if (cap_status == cudaStreamCaptureStatusNone) cudaEventSynchronize(bs->uploaded);
  std::memcpy(bs->staging, d.data(), sizeof(BatchScene) * n);
  if (cudaMemcpyAsync(bs->desc, bs->staging, sizeof(BatchScene) * n, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaEventRecord(bs->uploaded, stream) != cudaSuccess) {
    err = "upload of backward descriptors failed";
    return PIKO_ERR_CUDA;
  }
  BatchBwdParams p;
  p.n = n;
  p.sc = bs->params.sc;
  p.btile_prefix = bs->params.btile_prefix;
  p.total_btiles = bs->params.total_btiles;
  p.vtx = bs->vtx;
  p.invw = bs->params.invw;  // the interpolation of the last forward_batch
  static int per_sm_of[64] = {0};  // the shared-memory opt-in is per device
  int dev = 0;
  cudaGetDevice(&dev);
  int& per_sm = per_sm_of[dev & 63];
  if (per_sm == 0) {
    int v = 0;
    // both instances share the launch bounds and the shared-memory size
    if (cudaFuncSetAttribute(k_batch_backward<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BATCH_BWD_SMEM) != cudaSuccess ||
        cudaFuncSetAttribute(k_batch_backward<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)BATCH_BWD_SMEM) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_batch_backward<false>, BWD_THREADS, BATCH_BWD_SMEM) !=
            cudaSuccess ||
        v < 1)
      v = 1;
    per_sm = v;
  }
  long long blocks = (long long)per_sm * num_sms;
  const long long need = (p.total_btiles + BATCH_BWD_WARPS - 1) / BATCH_BWD_WARPS;  // a tile per warp
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  if (bs->persp)
    k_batch_backward<true><<<(int)blocks, BWD_THREADS, BATCH_BWD_SMEM, stream>>>(p);
  else
    k_batch_backward<false><<<(int)blocks, BWD_THREADS, BATCH_BWD_SMEM, stream>>>(p);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    err = std::string("batch backward launch: ") + cudaGetErrorString(e);
    return PIKO_ERR_CUDA;
  }
  return PIKO_OK;
}
