// piko_process.cu -- the per-tile Process stage for one scene.
//
// Tiles are handed to CTAs by one of three schedules (Sec. 4.3 / 5.2.2 of
// the Piko paper): DirectMap (static round robin over a persistent grid),
// LoadBalance (an atomic tile queue) or one CTA per tile; the work of a tile
// is process_tile() in piko_tile.cuh.
#include "piko_tile.cuh"

namespace piko {

__host__ __device__ inline TileScene scene_of(const ProcessParams& p) {
  TileScene sc;
  sc.g = p.g;
  sc.mode = p.mode;
  sc.unclamped = p.unclamped;
  sc.small_px = p.small_px;
  sc.slot_bits = p.slot_bits;
  sc.nslots = p.nslots;
  sc.rec_stride = p.rec_stride;
  sc.tri_base = 0;
  sc.tris = p.tris;
  sc.vtx = p.vtx;
  sc.color = p.color;
  sc.normal = p.normal;
  sc.light = p.light;
  sc.vdot = p.vdot;
  sc.invw = p.invw;
  sc.T = p.num_triangles;
  sc.clip_tris = p.clip_tris;
  sc.clip_orig = p.clip_orig;
  sc.pos = p.clip_tris ? reinterpret_cast<const float4*>(p.pos) : nullptr;
  sc.mvp = p.mvp;
  sc.key_out = p.key_out;
  sc.rgba_out = p.rgba_out;
  sc.gnorm_out = p.gnorm_out;
  sc.galb_out = p.galb_out;
  return sc;
}

#ifndef PIKO_PROCESS_MAXNREG
#define PIKO_PROCESS_MAXNREG 64
#endif
// The register cap trades spills on the static and dynamic schedules' tile
// loops for occupancy (about 120 registers uncapped); the one-CTA-per-tile
// instance fits 64 registers without spilling.
// One instance per schedule (SCHED = PIKO_SCHED_*), so that each carries
// only its own tile loop, per value of the work-counter option (STATS), so
// that the counters hold no registers when they are off, per attribute
// interpolation (PERSP: perspective-correct) and per clipping setting
// (CLIP: sub-triangles and clipped winners).  The scene is
// read in place from the grid-constant parameter block.
struct ProcessLaunch {
  ProcessParams p;
  TileScene sc;
};
template <int SCHED, bool STATS, bool PERSP, bool CLIP>
__global__ void __maxnreg__(PIKO_PROCESS_MAXNREG) k_process(const __grid_constant__ ProcessLaunch pl) {
  const ProcessParams& p = pl.p;
  extern __shared__ __align__(16) unsigned long long smem[];
  const int bin_px = 1 << (p.g.bshift_x + p.g.bshift_y);
  const int nt = blockDim.x, tid = threadIdx.x;
  __shared__ int s_tile[2];
  __shared__ unsigned s_nbig;
  TileSmem sm;
  sm.skey = smem;
  sm.sbig = reinterpret_cast<int*>(smem + bin_px);
  sm.sfrag = sm.sbig + nt;
  sm.srec = sm.sfrag + (nt >> 5) * FRAG_WARP_WORDS;
  sm.s_nbig = &s_nbig;
  const TileScene& sc = pl.sc;
  for (int i = tid; i < bin_px; i += nt) sm.skey[i] = KEY_EMPTY;
  pdl_wait();  // bin lists and status of the scatter pass
  // the first tile's range is loaded before the status word is tested, so
  // that the two global round trips overlap (static and hardware schedules)
  unsigned nbeg = 0u, nend = 0u;
  if (SCHED != PIKO_SCHED_DYNAMIC && (int)blockIdx.x < p.ntiles) {
    nbeg = __ldg(p.bin_off + blockIdx.x);
    nend = __ldg(p.bin_off + blockIdx.x + 1);
  }
  if (p.st->flags & STATUS_SKIP_MASK) return;
  constexpr bool dynamic = SCHED == PIKO_SCHED_DYNAMIC;
  if (tid == 0) {
    s_nbig = 0u;
    if (dynamic) s_tile[0] = (int)atomicAdd(&p.st->queue_head, 1u);
  }
  __syncthreads();
  unsigned big_base = 0u;
  TileStats st = {0ull, 0ull, 0ull};
  for (int iter = 0;; ++iter) {
    int tile;
    if (SCHED == PIKO_SCHED_HARDWARE) {
      if (iter > 0) break;
      tile = blockIdx.x;
    } else if (SCHED == PIKO_SCHED_STATIC) {
      tile = blockIdx.x + iter * gridDim.x;
    } else {
      tile = s_tile[iter & 1];
      // fetch the next tile now; it is read after the tile's closing barrier
      if (tid == 0 && tile < p.ntiles) s_tile[(iter + 1) & 1] = (int)atomicAdd(&p.st->queue_head, 1u);
    }
    if (tile >= p.ntiles) break;
    unsigned beg, end;
    if (SCHED == PIKO_SCHED_DYNAMIC) {
      beg = __ldg(p.bin_off + tile);
      end = __ldg(p.bin_off + tile + 1);
    } else {
      beg = nbeg;
      end = nend;
      // the static schedule's next tile is known: its range loads during this one
      const int next = tile + (int)gridDim.x;
      if (SCHED == PIKO_SCHED_STATIC && next < p.ntiles) {
        nbeg = __ldg(p.bin_off + next);
        nend = __ldg(p.bin_off + next + 1);
      }
    }
    process_tile<STATS, PERSP, CLIP>(sc, tile, beg, end, p.bin_tris, sm, big_base, st);
  }
  if (STATS) {  // one atomic per warp: same-address atomics from every thread serialise
    for (int o = 16; o > 0; o >>= 1) {
      st.tests += __shfl_down_sync(FULL_MASK, st.tests, o);
      st.frags += __shfl_down_sync(FULL_MASK, st.frags, o);
      st.shaded += __shfl_down_sync(FULL_MASK, st.shaded, o);
    }
    if ((tid & 31) == 0) {
      atomicAdd(&p.st->tests, st.tests);
      atomicAdd(&p.st->frags, st.frags);
      atomicAdd(&p.st->shaded, st.shaded);
    }
  }
}

// ---------------------------------------------------------------- host side
static void layout(ProcessParams& p, int threads) {
  (void)threads;
  tile_layout(p.num_triangles, 1 << (p.g.bshift_x + p.g.bshift_y), p.mode, p.color != nullptr, p.invw != nullptr, 511,
              p.slot_bits, p.nslots, p.rec_stride, p.slots_hint);
}

static size_t smem_bytes(const ProcessParams& p, int threads) {
  return tile_smem_bytes(1 << (p.g.bshift_x + p.g.bshift_y), threads, p.nslots, p.rec_stride);
}

using ProcessKernel = void (*)(ProcessLaunch);

template <bool STATS, bool PERSP, bool CLIP>
static ProcessKernel process_kernel_of(int schedule) {
  if (schedule == PIKO_SCHED_DYNAMIC) return k_process<PIKO_SCHED_DYNAMIC, STATS, PERSP, CLIP>;
  if (schedule == PIKO_SCHED_HARDWARE) return k_process<PIKO_SCHED_HARDWARE, STATS, PERSP, CLIP>;
  return k_process<PIKO_SCHED_STATIC, STATS, PERSP, CLIP>;
}

template <bool CLIP>
static ProcessKernel process_kernel_clip(const ProcessParams& p) {
  if (p.invw)
    return p.stats ? process_kernel_of<true, true, CLIP>(p.schedule) : process_kernel_of<false, true, CLIP>(p.schedule);
  return p.stats ? process_kernel_of<true, false, CLIP>(p.schedule) : process_kernel_of<false, false, CLIP>(p.schedule);
}

static ProcessKernel process_kernel(const ProcessParams& p) {
  return p.clip_tris ? process_kernel_clip<true>(p) : process_kernel_clip<false>(p);
}

cudaError_t process_occupancy(const ProcessParams& p0, int threads, int* blocks_per_sm) {
  ProcessParams p = p0;
  layout(p, threads);
  const size_t smem = smem_bytes(p, threads);
  const ProcessKernel k = process_kernel(p);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem);
}

cudaError_t launch_process(const ProcessParams& p0, int threads, int grid, cudaStream_t s) {
  ProcessParams p = p0;
  layout(p, threads);
  const size_t smem = smem_bytes(p, threads);
  const ProcessKernel k = process_kernel(p);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  ProcessLaunch pl;
  pl.p = p;
  pl.sc = scene_of(p);
  const cudaError_t e = launch_pdl(k, grid, threads, smem, s, pl);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace piko
