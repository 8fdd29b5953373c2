// piko_noalloc.cu -- a forward pass for callers that may not allocate GPU memory.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA stream
// capture that must not grow the graph's memory footprint, plugins hosted by
// an application that owns the device allocator (or forbids device
// allocation after start-up), and real-time loops where an allocation, with
// its implicit synchronisation, would break the frame budget.  For them,
// piko_raster_forward_noalloc runs the same kernels as piko_raster_forward
// with every scratch buffer carved out of one fixed array below, so it needs
// no handle and calls no allocator.  The caller still supplies the scene and
// the framebuffer.
//
// Limits: at most PIKO_NOALLOC_MAX_VERTICES vertices, PIKO_NOALLOC_MAX_TRIANGLES
// triangles, PIKO_NOALLOC_MAX_BINS tiles and PIKO_NOALLOC_MAX_BIN_ENTRIES
// (triangle, tile) pairs; about 6.3 MB of device memory that every GPU which
// loads this library keeps until the process exits.
#include <cuda.h>

#include <atomic>
#include <mutex>

#include "piko_internal.cuh"
#include "piko_scan.cuh"

using namespace piko;

namespace {

constexpr size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// layout of the scratch array
// The scan's chunk states sit directly before the per-tile counts so that
// one memset clears both at the start of every call.
constexpr int MAX_CHUNKS = 64;
constexpr size_t OFF_STATUS = 0;
constexpr size_t OFF_VTX = align256(OFF_STATUS + sizeof(DevStatus));
constexpr size_t OFF_VDOT = align256(OFF_VTX + sizeof(int4) * PIKO_NOALLOC_MAX_VERTICES);
constexpr size_t OFF_RECT = align256(OFF_VDOT + sizeof(float) * PIKO_NOALLOC_MAX_VERTICES);
constexpr size_t OFF_CHUNKS = align256(OFF_RECT + sizeof(BinRect) * PIKO_NOALLOC_MAX_TRIANGLES);
constexpr size_t OFF_COUNT = OFF_CHUNKS + sizeof(unsigned long long) * MAX_CHUNKS;
constexpr size_t OFF_OFFS = align256(OFF_COUNT + sizeof(unsigned) * 2 * PIKO_NOALLOC_MAX_BINS);
constexpr size_t OFF_CURSOR = align256(OFF_OFFS + sizeof(unsigned) * (PIKO_NOALLOC_MAX_BINS + 1));
constexpr size_t OFF_ENTRIES = align256(OFF_CURSOR + sizeof(unsigned) * PIKO_NOALLOC_MAX_BINS);
static_assert(PIKO_NOALLOC_MAX_BINS / FWD_SCAN_CHUNK + 1 <= MAX_CHUNKS, "scan chunk states must fit");
static_assert(OFF_COUNT % 256 == 0, "counts stay 256-byte aligned");
constexpr size_t SCRATCH_BYTES = align256(OFF_ENTRIES + sizeof(unsigned) * (size_t)PIKO_NOALLOC_MAX_BIN_ENTRIES);

// The one scratch buffer shared by every call on a device.  In host code this
// name is only a stand-in for the device symbol, never a device address: the
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

std::atomic<unsigned> g_scan_epoch{0};
std::mutex g_setup_lock;

// The array's device address belongs to the module instance of one CUDA
// context: the primary context of a device normally, but a caller may run
// in a context of its own (cuCtxCreate), and cudaDeviceReset replaces the
// primary context.  So the address is cached per context, keyed by the
// context's unique id (cuCtxGetId: never reused within a process), and
// looked up again for a context not seen before.  The two driver calls are
// reached through the runtime's entry-point query, so the library does not
// link the driver library directly.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
constexpr int MAX_CONTEXTS = 64;
struct CtxScratch {
  unsigned long long ctx_id;
  unsigned char* addr;
};
CtxScratch g_ctx_cache[MAX_CONTEXTS] = {};
int g_ctx_count = 0, g_ctx_next = 0;

bool driver_entry_points() {
  if (g_ctx_get_current && g_ctx_get_id) return true;
  cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
  void* f1 = nullptr;
  void* f2 = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
      cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
      q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
    cudaGetLastError();
    return false;
  }
  g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
  g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  return true;
}

// Device address of the scratch array in the current context.  The first
// call in a context (once per device for callers on the primary context)
// looks it up with cudaGetSymbolAddress; later calls reuse it.
int scratch_for_current_context(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
    cudaGetLastError();
    return PIKO_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_lock);
  if (!driver_entry_points()) return PIKO_ERR_CUDA;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return PIKO_ERR_CUDA;
  if (!ctx) {
    // no context is current on this thread yet: the runtime would use the
    // device's primary context, so make that one current and key on it
    if (cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      return PIKO_ERR_CUDA;
    }
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return PIKO_ERR_CUDA;
  }
  if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return PIKO_ERR_CUDA;
  for (int i = 0; i < g_ctx_count; ++i)
    if (g_ctx_cache[i].ctx_id == id) {
      *out = g_ctx_cache[i].addr;
      return PIKO_OK;
    }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return PIKO_ERR_CUDA;
  }
  // a context that is gone keeps its entry until the ring wraps; ids are
  // never reused, so a stale entry is never matched
  CtxScratch& slot = g_ctx_count < MAX_CONTEXTS ? g_ctx_cache[g_ctx_count++] : g_ctx_cache[g_ctx_next++ % MAX_CONTEXTS];
  slot.ctx_id = id;
  slot.addr = static_cast<unsigned char*>(p);
  *out = slot.addr;
  return PIKO_OK;
}

bool valid_bin(int b) { return b == 8 || b == 16 || b == 32 || b == 64; }
int ilog2(int v) {
  int s = 0;
  while ((1 << s) < v) ++s;
  return s;
}
bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int piko_raster_forward_noalloc(const piko_scene* s, piko_framebuffer* fb, int bin_w, int bin_h,
                                           int schedule, int32_t* status_out, void* cuda_stream) {
  // ---- host-side argument checks: nothing is enqueued when one fails
  if (!s || !fb || !fb->key) return PIKO_ERR_INVALID_ARG;
  if (s->width < 1 || s->height < 1 || s->width > 32767 || s->height > 32767) return PIKO_ERR_INVALID_ARG;
  if (!valid_bin(bin_w) || !valid_bin(bin_h)) return PIKO_ERR_INVALID_ARG;
  if (schedule < PIKO_SCHED_STATIC || schedule > PIKO_SCHED_HARDWARE) return PIKO_ERR_INVALID_ARG;
  if (s->num_vertices < 0 || s->num_triangles < 0 || s->num_vertices > PIKO_NOALLOC_MAX_VERTICES ||
      s->num_triangles > PIKO_NOALLOC_MAX_TRIANGLES)
    return PIKO_ERR_INVALID_ARG;
  const int nbx = (s->width + bin_w - 1) / bin_w, nby = (s->height + bin_h - 1) / bin_h;
  if ((long long)nbx * nby > PIKO_NOALLOC_MAX_BINS) return PIKO_ERR_INVALID_ARG;
  if (s->num_vertices > 0 && (!s->pos || !aligned16(s->pos))) return PIKO_ERR_INVALID_ARG;
  if (s->num_triangles > 0 && (!s->tris || !aligned16(s->tris))) return PIKO_ERR_INVALID_ARG;
  if (s->shade_mode < PIKO_SHADE_GOURAUD || s->shade_mode > PIKO_SHADE_GBUFFER || s->reserved != 0)
    return PIKO_ERR_INVALID_ARG;
  if (s->num_triangles > 0 && s->shade_mode == PIKO_SHADE_GOURAUD && !s->color) return PIKO_ERR_INVALID_ARG;
  if (s->num_triangles > 0 && s->shade_mode != PIKO_SHADE_GOURAUD && !s->normal) return PIKO_ERR_INVALID_ARG;
  if (s->shade_mode == PIKO_SHADE_LAMBERT && !s->light_dir) return PIKO_ERR_INVALID_ARG;
  if (s->shade_mode == PIKO_SHADE_GBUFFER && (!fb->gbuf_normal || !fb->gbuf_albedo)) return PIKO_ERR_INVALID_ARG;

  unsigned char* base = nullptr;
  int r = scratch_for_current_context(&base);
  if (r != PIKO_OK) return r;
  int dev = 0, num_sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return PIKO_ERR_CUDA;
  }
  DevStatus* status = reinterpret_cast<DevStatus*>(base + OFF_STATUS);
  int4* vtx = reinterpret_cast<int4*>(base + OFF_VTX);
  float* vdot = reinterpret_cast<float*>(base + OFF_VDOT);
  BinRect* rect = reinterpret_cast<BinRect*>(base + OFF_RECT);
  unsigned* bin_count = reinterpret_cast<unsigned*>(base + OFF_COUNT);
  unsigned* bin_off = reinterpret_cast<unsigned*>(base + OFF_OFFS);
  unsigned* cursor = reinterpret_cast<unsigned*>(base + OFF_CURSOR);
  unsigned* bin_tris = reinterpret_cast<unsigned*>(base + OFF_ENTRIES);
  unsigned long long* chunk_state = reinterpret_cast<unsigned long long*>(base + OFF_CHUNKS);

  RasterGeom g;
  g.W = s->width; g.H = s->height;
  g.bshift_x = ilog2(bin_w); g.bshift_y = ilog2(bin_h);
  g.nbx = nbx; g.nby = nby;
  const int nbins = nbx * nby;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

  // The array keeps whatever the previous call left in it: the status word,
  // the scan's chunk states and the per-tile counts must start at zero.  A
  // cleared chunk state reads as "not published", so no state left by an
  // earlier call (with more tiles, or an epoch tag that has wrapped) can be
  // taken for this call's.
  if (cudaMemsetAsync(status, 0, sizeof(DevStatus), st) != cudaSuccess ||
      cudaMemsetAsync(chunk_state, 0, (OFF_COUNT - OFF_CHUNKS) + sizeof(unsigned) * 2 * nbins, st) != cudaSuccess) {
    cudaGetLastError();
    return PIKO_ERR_CUDA;
  }
  const bool lambert = s->shade_mode == PIKO_SHADE_LAMBERT;
  launch_vertex(g.W, g.H, s->num_vertices, s->pos, s->mvp, vtx, lambert ? s->normal : nullptr, s->light_dir,
                lambert ? vdot : nullptr, nullptr, num_sms, st);
  launch_setup_count(g, s->num_triangles, s->tris, s->num_vertices, vtx, rect, bin_count, status, 0, num_sms, st);
  launch_scan(nbins, bin_count, bin_off, cursor, (unsigned long long)PIKO_NOALLOC_MAX_BIN_ENTRIES, status, chunk_state,
              ++g_scan_epoch, st);
  launch_scatter(g, s->num_triangles, rect, bin_off, cursor, bin_tris, (unsigned long long)PIKO_NOALLOC_MAX_BIN_ENTRIES,
                 status, num_sms, st);

  ProcessParams p;
  p.slots_hint = 0;
  p.g = g;
  p.ntiles = nbins;
  p.schedule = schedule;
  p.small_px = 32;
  p.mode = s->shade_mode;
  p.unclamped = 0;
  p.stats = 0;
  p.num_triangles = s->num_triangles;
  p.tris = s->tris;
  p.vtx = vtx;
  p.color = s->color;
  p.normal = s->normal;
  p.light = s->light_dir;
  p.vdot = vdot;
  p.invw = nullptr;  // screen-space attributes only
  p.clip_tris = nullptr;  // no clipping: out-of-range vertices cull their triangles
  p.clip_orig = nullptr;
  p.pos = s->pos;
  p.mvp = s->mvp;
  p.bin_off = bin_off;
  p.bin_tris = bin_tris;
  p.key_out = reinterpret_cast<unsigned long long*>(fb->key);
  p.rgba_out = reinterpret_cast<float4*>(fb->rgba);
  p.gnorm_out = reinterpret_cast<uint2*>(fb->gbuf_normal);
  p.galb_out = reinterpret_cast<uint2*>(fb->gbuf_albedo);
  p.st = status;
  const int threads = default_process_threads(bin_w * bin_h, nbins, num_sms);
  int grid = nbins;
  if (schedule != PIKO_SCHED_HARDWARE) {
    int per_sm = 0;
    if (process_occupancy(p, threads, &per_sm) != cudaSuccess) {
      cudaGetLastError();
      return PIKO_ERR_CUDA;
    }
    if (per_sm < 1) per_sm = 1;
    grid = per_sm * num_sms < nbins ? per_sm * num_sms : nbins;
  }
  if (launch_process(p, threads, grid, st) != cudaSuccess) return PIKO_ERR_CUDA;
  if (status_out && cudaMemcpyAsync(status_out, &status->first_code, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                    st) != cudaSuccess) {
    cudaGetLastError();
    return PIKO_ERR_CUDA;
  }
  return PIKO_OK;
}
