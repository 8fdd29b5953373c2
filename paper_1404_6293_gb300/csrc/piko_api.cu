// piko_api.cu -- the C ABI: handles, scratch memory, argument checks, launch order.
#include <stdio.h>
#include <string.h>

#include <string>

#include "piko_internal.cuh"
#include "piko_scan.cuh"

using namespace piko;

struct BatchState;
void batch_state_free(BatchState* bs);
int batch_prepare(BatchState*& bs, int num_sms, const piko_scene* scenes, int n, piko_framebuffer* fbs,
                  const int32_t* bin_sizes, const int32_t* schedules, int default_bin_w, int default_bin_h,
                  int default_schedule, int unclamped, int persp, cudaStream_t stream, std::string& err);
int batch_launch_forward(BatchState* bs, DevStatus* st, bool persistent, cudaStream_t stream, std::string& err,
                         long long wait_budget, int withhold);
long long batch_capacity(const BatchState* bs);
void batch_note_entries(BatchState* bs, long long entries);
int batch_grow_entries(BatchState* bs, long long need, std::string& err);
int batch_launch_backward(BatchState* bs, const piko_scene* scenes, int n, const piko_framebuffer* fbs,
                          const float* const* dl, float* const* dc, float* const* dn, float* const* dlt, int num_sms,
                          cudaStream_t stream, std::string& err);

int piko_backward_launch(int W, int H, int mode, int unclamped, int T, int V, const int* tris, const int4* vtx,
                         const float* color, const float* normal, const float* light, const float* invw,
                         const float* pos, const float* mvp, const unsigned long long* key,
                         const float* dl_drgba, float* dcolor, float* dnormal, float* dlight, int num_sms,
                         cudaStream_t s);

struct piko_raster {
  int W, H, bin_w, bin_h, schedule;
  RasterGeom g;
  int nbins;
  int threads = 256;
  int unclamped = 0;
  int perspective = 0;  // perspective-correct attributes (single-scene calls)
  int check_capacity = 1;
  int small_px = 32;
  int stats = 0;
  int batch_launch = 0;  // 0 persistent cooperative, 1 one launch per phase
  int clip = 0;                      // near/far clipping instead of culling (PIKO_OPT_CLIP)
  int exact_bins = 0;                // exact triangle-vs-bin overlap in AssignBin (PIKO_OPT_EXACT_BINS)
  long long wait_budget = 40000000;  // clock cycles a device-side wait may take (PIKO_OPT_WAIT_BUDGET)
  int withhold = 0;                  // test hooks (PIKO_OPT_TEST_WITHHOLD)
  BatchState* batch = nullptr;
  cudaEvent_t stage_ev[PIKO_NUM_STAGE_EVENTS] = {};
  bool use_stage_ev = false;
  int device = 0, num_sms = 0;
  // scratch (device)
  int4* vtx = nullptr;
  long long vcap = 0;
  float* vdot = nullptr;  // n . L per vertex for Lambert
  long long dcap = 0;
  float* invw = nullptr;  // 1 / clip w per vertex, with perspective-correct attributes
  long long icap = 0;
  BinRect* rect = nullptr;
  long long tcap = 0;
  unsigned* bin_count = nullptr;  // 2 * nbins, zero between frames
  unsigned* bin_off = nullptr;    // nbins + 1
  unsigned* cursor = nullptr;
  unsigned long long* chunk_state = nullptr;  // look-back state of the scan
  unsigned scan_epoch = 0;
  unsigned* bin_tris = nullptr;
  long long ecap = 0;
  // AssignBin's list of heavy triangles (chunks of (triangle, bin) pairs
  // spread over whole CTAs), and the count pass's parity
  uint2* heavy = nullptr;
  unsigned heavy_epoch = 0;
  // fragment buffers of the unfused pipeline (PIKO_SCHED_UNFUSED)
  unsigned* frag_pix = nullptr;
  unsigned long long* frag_key = nullptr;
  float4* frag_rgba = nullptr;
  long long fcap_pix = 0, fcap_key = 0, fcap_rgba = 0;
  unsigned* h_frags = nullptr;  // pinned: fragment count read back
  // near/far clipping: sub-triangles (3 snapped points each) and their triangle
  int4* clip_tris = nullptr;
  unsigned* clip_orig = nullptr;
  long long ccap_tris = 0, ccap_orig = 0;
  unsigned* h_clips = nullptr;  // pinned: sub-triangle count read back
  // device copies of a scene and framebuffer held in host memory (piko_raster_forward_host)
  float4* hs_pos = nullptr;
  int* hs_tris = nullptr;
  float* hs_color = nullptr;
  float* hs_normal = nullptr;
  float* hs_small = nullptr;  // mvp [16] then light [3]
  unsigned long long* hs_key = nullptr;
  float4* hs_rgba = nullptr;
  uint2* hs_gn = nullptr;
  uint2* hs_ga = nullptr;
  long long hcap_pos = 0, hcap_tris = 0, hcap_color = 0, hcap_normal = 0, hcap_small = 0, hcap_key = 0,
            hcap_rgba = 0, hcap_gn = 0, hcap_ga = 0;
  DevStatus* status = nullptr;
  unsigned long long* h_needed = nullptr;  // pinned
  long long last_entries = 0;              // bin entries of the last frame read back (0: none yet)
  cudaStream_t last_stream = nullptr;
  std::string err;
};

namespace {

int fail(piko_raster* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(piko_raster* h, cudaError_t e, const char* where) {
  return fail(h, PIKO_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

int ilog2(int v) {
  int s = 0;
  while ((1 << s) < v) ++s;
  return s;
}

bool valid_bin(int b) { return b == 8 || b == 16 || b == 32 || b == 64; }

template <typename T>
int grow(piko_raster* h, T** ptr, long long* cap, long long need, const char* what) {
  if (need <= *cap) return PIKO_OK;
  long long n = need + need / 4 + 1024;
  if (*ptr) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceSynchronize");
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
  }
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), (size_t)n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, PIKO_ERR_OOM, std::string("cudaMalloc of ") + what + " failed");
  }
  *cap = n;
  return PIKO_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

int piko_raster_version(void) { return 100; }

piko_raster* piko_raster_create(int width, int height, int bin_w, int bin_h, int schedule) {
  if (width < 1 || height < 1 || width > 32767 || height > 32767) return nullptr;
  if (!valid_bin(bin_w) || !valid_bin(bin_h)) return nullptr;
  if (schedule < PIKO_SCHED_STATIC || schedule > PIKO_SCHED_UNFUSED) return nullptr;
  piko_raster* h = new piko_raster();
  h->W = width; h->H = height; h->bin_w = bin_w; h->bin_h = bin_h; h->schedule = schedule;
  h->g.W = width; h->g.H = height;
  h->g.bshift_x = ilog2(bin_w); h->g.bshift_y = ilog2(bin_h);
  h->g.nbx = (width + bin_w - 1) / bin_w;
  h->g.nby = (height + bin_h - 1) / bin_h;
  h->nbins = h->g.nbx * h->g.nby;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return nullptr;
  }
  h->threads = default_process_threads(bin_w * bin_h, h->nbins, h->num_sms);
  bool ok = cudaMalloc(&h->bin_count, sizeof(unsigned) * 2 * h->nbins) == cudaSuccess &&
            cudaMalloc(&h->bin_off, sizeof(unsigned) * (h->nbins + 1)) == cudaSuccess &&
            cudaMalloc(&h->cursor, sizeof(unsigned) * h->nbins) == cudaSuccess &&
            cudaMalloc(&h->chunk_state, sizeof(unsigned long long) * scan_chunks(h->nbins)) == cudaSuccess &&
            cudaMemset(h->chunk_state, 0, sizeof(unsigned long long) * scan_chunks(h->nbins)) == cudaSuccess &&
            cudaMalloc(&h->status, sizeof(DevStatus)) == cudaSuccess &&
            cudaMalloc(&h->heavy, sizeof(uint2) * HEAVY_LIST_CAP) == cudaSuccess &&
            cudaMallocHost(&h->h_needed, sizeof(unsigned long long)) == cudaSuccess &&
            cudaMallocHost(&h->h_frags, sizeof(unsigned)) == cudaSuccess &&
            cudaMallocHost(&h->h_clips, sizeof(unsigned)) == cudaSuccess &&
            cudaMemset(h->bin_count, 0, sizeof(unsigned) * 2 * h->nbins) == cudaSuccess &&
            cudaMemset(h->status, 0, sizeof(DevStatus)) == cudaSuccess &&
            cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    piko_raster_destroy(h);
    return nullptr;
  }
  return h;
}

void piko_raster_destroy(piko_raster* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  cudaFree(h->vtx);
  cudaFree(h->vdot);
  cudaFree(h->invw);
  cudaFree(h->rect);
  cudaFree(h->bin_count);
  cudaFree(h->bin_off);
  cudaFree(h->cursor);
  cudaFree(h->chunk_state);
  cudaFree(h->bin_tris);
  cudaFree(h->heavy);
  cudaFree(h->frag_pix);
  cudaFree(h->frag_key);
  cudaFree(h->frag_rgba);
  cudaFree(h->clip_tris);
  cudaFree(h->clip_orig);
  cudaFree(h->hs_pos);
  cudaFree(h->hs_tris);
  cudaFree(h->hs_color);
  cudaFree(h->hs_normal);
  cudaFree(h->hs_small);
  cudaFree(h->hs_key);
  cudaFree(h->hs_rgba);
  cudaFree(h->hs_gn);
  cudaFree(h->hs_ga);
  cudaFree(h->status);
  batch_state_free(h->batch);
  if (h->h_needed) cudaFreeHost(h->h_needed);
  if (h->h_frags) cudaFreeHost(h->h_frags);
  if (h->h_clips) cudaFreeHost(h->h_clips);
  cudaGetLastError();
  delete h;
}

const char* piko_raster_last_error(const piko_raster* h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

// Chunks the heavy-triangle list may hold: none under test hook bit 2, so
// that every heavy triangle takes the path of a full list.
static unsigned heavy_cap(const piko_raster* h) { return (h->withhold & TEST_WITHHOLD_HEAVY) ? 0u : HEAVY_LIST_CAP; }

int piko_raster_set_option(piko_raster* h, int key, int value) {
  if (!h) return PIKO_ERR_INVALID_ARG;
  switch (key) {
    case PIKO_OPT_THREADS_PER_TILE:
      if (value != 64 && value != 128 && value != 256 && value != 512)
        return fail(h, PIKO_ERR_INVALID_ARG, "threads per tile must be 64, 128, 256 or 512");
      h->threads = value;
      return PIKO_OK;
    case PIKO_OPT_UNCLAMPED:
      if (value != 0 && value != 1) return fail(h, PIKO_ERR_INVALID_ARG, "unclamped must be 0 or 1");
      h->unclamped = value;
      return PIKO_OK;
    case PIKO_OPT_CHECK_CAPACITY:
      if (value != 0 && value != 1) return fail(h, PIKO_ERR_INVALID_ARG, "check_capacity must be 0 or 1");
      h->check_capacity = value;
      return PIKO_OK;
    case PIKO_OPT_SCHEDULE:
      if (value < PIKO_SCHED_STATIC || value > PIKO_SCHED_UNFUSED)
        return fail(h, PIKO_ERR_INVALID_ARG, "unknown schedule");
      h->schedule = value;
      return PIKO_OK;
    case PIKO_OPT_STATS:
      if (value != 0 && value != 1) return fail(h, PIKO_ERR_INVALID_ARG, "stats must be 0 or 1");
      h->stats = value;
      return PIKO_OK;
    case PIKO_OPT_BATCH_LAUNCH:
      if (value != 0 && value != 1) return fail(h, PIKO_ERR_INVALID_ARG, "batch launch must be 0 or 1");
      h->batch_launch = value;
      return PIKO_OK;
    case PIKO_OPT_PERSPECTIVE:
      if (value != 0 && value != 1) return fail(h, PIKO_ERR_INVALID_ARG, "perspective must be 0 or 1");
      h->perspective = value;
      return PIKO_OK;
    case PIKO_OPT_CLIP:
      if (value != 0 && value != 1) return fail(h, PIKO_ERR_INVALID_ARG, "clip must be 0 or 1");
      h->clip = value;
      return PIKO_OK;
    case PIKO_OPT_EXACT_BINS:
      if (value != 0 && value != 1) return fail(h, PIKO_ERR_INVALID_ARG, "exact bins must be 0 or 1");
      h->exact_bins = value;
      return PIKO_OK;
    case PIKO_OPT_WAIT_BUDGET:
      if (value < 1 || value > 1000000) return fail(h, PIKO_ERR_INVALID_ARG, "wait budget must be 1..1000000 kcycles");
      h->wait_budget = (long long)value * 1000;
      return PIKO_OK;
    case PIKO_OPT_TEST_WITHHOLD:
      if (value < 0 || value > 7) return fail(h, PIKO_ERR_INVALID_ARG, "withhold must be 0..7");
      h->withhold = value;
      return PIKO_OK;
    case PIKO_OPT_SMALL_TRI_PIXELS:
      if (value < 0 || value > 4096) return fail(h, PIKO_ERR_INVALID_ARG, "small-triangle pixels out of range");
      h->small_px = value;
      return PIKO_OK;
    default:
      return fail(h, PIKO_ERR_INVALID_ARG, "unknown option");
  }
}

int piko_raster_reserve(piko_raster* h, int64_t max_vertices, int64_t max_triangles, int64_t max_bin_entries) {
  if (!h) return PIKO_ERR_INVALID_ARG;
  if (max_vertices < 0 || max_triangles < 0 || max_bin_entries < 0 || max_vertices > INT32_MAX ||
      max_triangles > INT32_MAX || max_bin_entries > 0xFFFFFFF0LL)
    return fail(h, PIKO_ERR_INVALID_ARG, "reserve sizes out of range");
  int r;
  if ((r = grow(h, &h->vtx, &h->vcap, max_vertices, "vertex buffer")) != PIKO_OK) return r;
  if ((r = grow(h, &h->vdot, &h->dcap, max_vertices, "vertex light terms")) != PIKO_OK) return r;
  // 1/w too, so that turning perspective-correct attributes on later needs no allocation
  if ((r = grow(h, &h->invw, &h->icap, max_vertices, "vertex 1/w")) != PIKO_OK) return r;
  if ((r = grow(h, &h->rect, &h->tcap, max_triangles, "bin rectangles")) != PIKO_OK) return r;
  if ((r = grow(h, &h->bin_tris, &h->ecap, max_bin_entries, "bin lists")) != PIKO_OK) return r;
  cudaError_t e = cudaDeviceSynchronize();
  return e == cudaSuccess ? PIKO_OK : cuda_fail(h, e, "reserve");
}

int piko_raster_status(piko_raster* h, int64_t* needed_bin_entries) {
  if (!h) return PIKO_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
  DevStatus st;
  e = cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "status read");
  e = cudaMemset(h->status, 0, sizeof(unsigned) * 2);  // flags and first_code only
  if (e != cudaSuccess) return cuda_fail(h, e, "status clear");
  if (needed_bin_entries) *needed_bin_entries = (int64_t)st.needed;
  if (st.first_code != 0) {
    static const char* names[] = {"ok", "invalid argument", "cuda", "out of memory",
                                  "bin lists overflowed their capacity", "device wait timed out",
                                  "triangle index outside [0, V)"};
    h->err = st.first_code < 7 ? names[st.first_code] : "device error";
  }
  return (int)st.first_code;
}

static int check_scene(piko_raster* h, const piko_scene* s) {
  if (!s) return fail(h, PIKO_ERR_INVALID_ARG, "scene is NULL");
  if (s->width != h->W || s->height != h->H)
    return fail(h, PIKO_ERR_INVALID_ARG, "scene size differs from the rasterizer's");
  if (s->num_vertices < 0 || s->num_triangles < 0) return fail(h, PIKO_ERR_INVALID_ARG, "negative counts");
  if (s->num_vertices > 0 && (!s->pos || !aligned16(s->pos)))
    return fail(h, PIKO_ERR_INVALID_ARG, "pos must be a 16-byte aligned device pointer");
  if (s->num_triangles > 0 && (!s->tris || !aligned16(s->tris)))
    return fail(h, PIKO_ERR_INVALID_ARG, "tris must be a 16-byte aligned device pointer");
  if (s->shade_mode < PIKO_SHADE_GOURAUD || s->shade_mode > PIKO_SHADE_GBUFFER)
    return fail(h, PIKO_ERR_INVALID_ARG, "unknown shade mode");
  if (s->shade_mode == PIKO_SHADE_GOURAUD && !s->color && s->num_triangles > 0)
    return fail(h, PIKO_ERR_INVALID_ARG, "Gouraud shading needs per-vertex colours");
  if (s->shade_mode != PIKO_SHADE_GOURAUD && !s->normal && s->num_triangles > 0)
    return fail(h, PIKO_ERR_INVALID_ARG, "Lambert / G-buffer shading needs per-vertex normals");
  if (s->shade_mode == PIKO_SHADE_LAMBERT && !s->light_dir)
    return fail(h, PIKO_ERR_INVALID_ARG, "Lambert shading needs light_dir");
  if (s->reserved != 0) return fail(h, PIKO_ERR_INVALID_ARG, "reserved field must be 0");
  return PIKO_OK;
}

// Near/far clipping: the sub-triangle list for this frame.  With the
// capacity check the count is read back (one host sync) and the list grown
// and refilled once if it overflowed; without it an overflow is reported as
// PIKO_ERR_OVERFLOW and the frame writes nothing.
static int clip_pass(piko_raster* h, const piko_scene* s, cudaStream_t st) {
  const int T = s->num_triangles;
  long long want = T / 8 + 1024;
  int r;
  for (int attempt = 0;; ++attempt) {
    if (h->ccap_tris < 3 * want || h->ccap_orig < want) {
      if ((r = grow(h, &h->clip_tris, &h->ccap_tris, 3 * want, "clipped triangles")) != PIKO_OK ||
          (r = grow(h, &h->clip_orig, &h->ccap_orig, want, "clipped triangle indices")) != PIKO_OK)
        return r;
    }
    const long long cap = h->ccap_tris / 3 < h->ccap_orig ? h->ccap_tris / 3 : h->ccap_orig;
    cudaError_t e = cudaMemsetAsync(&h->status->clip_count, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(h, e, "clip count clear");
    launch_clip(h->W, h->H, T, s->tris, s->num_vertices, s->pos, s->mvp, h->vtx, h->clip_tris, h->clip_orig,
                (unsigned)cap, h->status, h->num_sms, st);
    if (!h->check_capacity) return PIKO_OK;
    e = cudaMemcpyAsync(h->h_clips, &h->status->clip_count, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "clip count read-back");
    const long long need = (long long)*h->h_clips;
    if (need <= cap) return PIKO_OK;
    if (attempt > 0) return fail(h, PIKO_ERR_OVERFLOW, "clipped triangle list too large");
    want = need + need / 8 + 1024;
    if ((e = cudaMemsetAsync(h->status, 0, sizeof(unsigned) * 2, st)) != cudaSuccess)
      return cuda_fail(h, e, "status clear");
  }
}

// The fused (no tiling) and unfused (one kernel per stage) mappings, after
// the vertex stage.  Stage events: 2 after the rasterizer, 3 after shading
// (fused: the per-pixel pass; unfused: the fragment shader), 4 after the
// depth test (unfused), 5 at the end.
static int forward_other_mapping(piko_raster* h, const piko_scene* s, piko_framebuffer* fb, cudaStream_t st,
                                 bool ev) {
  const bool unfused = h->schedule == PIKO_SCHED_UNFUSED;
  AltInputs in;
  in.W = h->W; in.H = h->H; in.T = s->num_triangles; in.V = s->num_vertices;
  in.mode = s->shade_mode; in.unclamped = h->unclamped;
  in.tris = s->tris; in.vtx = h->vtx; in.color = s->color; in.normal = s->normal; in.light = s->light_dir;
  in.invw = h->perspective ? h->invw : nullptr;
  in.key = reinterpret_cast<unsigned long long*>(fb->key);
  in.rgba = reinterpret_cast<float4*>(fb->rgba);
  in.gnorm = reinterpret_cast<uint2*>(fb->gbuf_normal);
  in.galb = reinterpret_cast<uint2*>(fb->gbuf_albedo);
  in.st = h->status;
  in.frag_pix = nullptr; in.frag_key = nullptr; in.frag_rgba = nullptr; in.frag_cap = 0;
  in.pos = s->pos; in.mvp = s->mvp;
  in.clip_tris = h->clip ? h->clip_tris : nullptr;
  in.clip_orig = h->clip ? h->clip_orig : nullptr;
  in.clip_cap = h->clip ? (unsigned)(h->ccap_tris < h->ccap_orig ? h->ccap_tris : h->ccap_orig) : 0u;
  const bool persp = h->perspective != 0;
  const size_t key_bytes = sizeof(unsigned long long) * (size_t)h->W * h->H;
  int r;
  cudaError_t e;
  if (!unfused) {
    if ((e = cudaMemsetAsync(fb->key, 0xFF, key_bytes, st)) != cudaSuccess) return cuda_fail(h, e, "key clear");
    if ((e = alt_stage(in, ALT_RASTER_MIN, persp, h->num_sms, st)) != cudaSuccess) return cuda_fail(h, e, "raster");
    if (ev) cudaEventRecord(h->stage_ev[2], st);
    if ((e = alt_stage(in, ALT_SHADE_PIXELS, persp, h->num_sms, st)) != cudaSuccess) return cuda_fail(h, e, "shade");
    if (ev) {
      cudaEventRecord(h->stage_ev[3], st);
      cudaEventRecord(h->stage_ev[4], st);
      cudaEventRecord(h->stage_ev[5], st);
    }
    return PIKO_OK;
  }
  // fragment buffers: at least two fragments per pixel or four per triangle
  long long want = 2LL * h->W * h->H;
  if (4LL * s->num_triangles > want) want = 4LL * s->num_triangles;
  want += 4096;
  for (int attempt = 0;; ++attempt) {
    if (h->fcap_key < want) {
      if ((r = grow(h, &h->frag_pix, &h->fcap_pix, want, "fragment pixels")) != PIKO_OK ||
          (r = grow(h, &h->frag_key, &h->fcap_key, want, "fragment keys")) != PIKO_OK ||
          (r = grow(h, &h->frag_rgba, &h->fcap_rgba, want, "fragment colours")) != PIKO_OK)
        return r;
    }
    const long long cap = h->fcap_key < h->fcap_pix ? (h->fcap_key < h->fcap_rgba ? h->fcap_key : h->fcap_rgba)
                                                    : (h->fcap_pix < h->fcap_rgba ? h->fcap_pix : h->fcap_rgba);
    in.frag_pix = h->frag_pix; in.frag_key = h->frag_key; in.frag_rgba = h->frag_rgba;
    in.frag_cap = (unsigned long long)cap;
    if ((e = cudaMemsetAsync(&h->status->frag_count, 0, sizeof(unsigned), st)) != cudaSuccess ||
        (e = cudaMemsetAsync(fb->key, 0xFF, key_bytes, st)) != cudaSuccess)
      return cuda_fail(h, e, "fragment count / key clear");
    if ((e = alt_stage(in, ALT_RASTER_EMIT, persp, h->num_sms, st)) != cudaSuccess) return cuda_fail(h, e, "raster");
    if (!h->check_capacity) break;
    e = cudaMemcpyAsync(h->h_frags, &h->status->frag_count, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "fragment count read-back");
    const long long need = (long long)*h->h_frags;
    if (need <= cap) break;
    if (attempt > 0) return fail(h, PIKO_ERR_OVERFLOW, "fragment buffer too large");
    want = need + need / 8 + 4096;
    // the rasterizer recorded an overflow: clear it and emit again
    if ((e = cudaMemsetAsync(h->status, 0, sizeof(unsigned) * 2, st)) != cudaSuccess)
      return cuda_fail(h, e, "status clear");
  }
  if (ev) cudaEventRecord(h->stage_ev[2], st);
  if ((e = alt_stage(in, ALT_FRAG_SHADE, persp, h->num_sms, st)) != cudaSuccess) return cuda_fail(h, e, "fragment shader");
  if (ev) cudaEventRecord(h->stage_ev[3], st);
  if ((e = alt_stage(in, ALT_FRAG_DEPTH, persp, h->num_sms, st)) != cudaSuccess) return cuda_fail(h, e, "depth test");
  if (ev) cudaEventRecord(h->stage_ev[4], st);
  if ((e = alt_stage(in, ALT_FRAG_COMPOSITE, persp, h->num_sms, st)) != cudaSuccess ||
      (e = alt_stage(in, ALT_CLEAR_EMPTY, persp, h->num_sms, st)) != cudaSuccess)
    return cuda_fail(h, e, "composite");
  if (ev) cudaEventRecord(h->stage_ev[5], st);
  return PIKO_OK;
}

int piko_raster_forward(piko_raster* h, const piko_scene* s, piko_framebuffer* fb, void* cuda_stream) {
  if (!h) return PIKO_ERR_INVALID_ARG;
  int r = check_scene(h, s);
  if (r != PIKO_OK) return r;
  if (!fb || !fb->key) return fail(h, PIKO_ERR_INVALID_ARG, "framebuffer key is required");
  if (s->shade_mode == PIKO_SHADE_GBUFFER && (!fb->gbuf_normal || !fb->gbuf_albedo))
    return fail(h, PIKO_ERR_INVALID_ARG, "G-buffer mode needs gbuf_normal and gbuf_albedo");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->last_stream = st;
  const int V = s->num_vertices, T = s->num_triangles;
  if ((r = grow(h, &h->vtx, &h->vcap, V, "vertex buffer")) != PIKO_OK) return r;
  const bool lambert = s->shade_mode == PIKO_SHADE_LAMBERT;
  if (lambert && (r = grow(h, &h->vdot, &h->dcap, V, "vertex light terms")) != PIKO_OK) return r;
  if (h->perspective && (r = grow(h, &h->invw, &h->icap, V, "vertex 1/w")) != PIKO_OK) return r;
  if ((r = grow(h, &h->rect, &h->tcap, T, "bin rectangles")) != PIKO_OK) return r;
  if (h->ecap == 0 && (r = grow(h, &h->bin_tris, &h->ecap, (long long)T * 2 + 4096, "bin lists")) != PIKO_OK)
    return r;

  const bool ev = h->use_stage_ev;
  h->use_stage_ev = false;
  if (ev) cudaEventRecord(h->stage_ev[0], st);
  if (h->stats) cudaMemsetAsync(&h->status->tests, 0, 4 * sizeof(unsigned long long), st);
  launch_vertex(h->W, h->H, V, s->pos, s->mvp, h->vtx, lambert ? s->normal : nullptr, s->light_dir,
                lambert ? h->vdot : nullptr, h->perspective ? h->invw : nullptr, h->num_sms, st);
  if (h->clip && (r = clip_pass(h, s, st)) != PIKO_OK) return r;
  const int4* clip_tris = h->clip ? h->clip_tris : nullptr;
  const unsigned clip_cap = h->clip ? (unsigned)(h->ccap_tris < h->ccap_orig ? h->ccap_tris : h->ccap_orig) : 0u;
  if (clip_cap && (r = grow(h, &h->rect, &h->tcap, (long long)T + clip_cap, "bin rectangles")) != PIKO_OK) return r;
  if (ev) cudaEventRecord(h->stage_ev[1], st);
  if (h->schedule == PIKO_SCHED_FUSED || h->schedule == PIKO_SCHED_UNFUSED)
    return forward_other_mapping(h, s, fb, st, ev);
  for (int attempt = 0;; ++attempt) {
    if (h->stats && attempt > 0) cudaMemsetAsync(&h->status->binned, 0, sizeof(unsigned long long), st);
    // a frame of one scan chunk of bins is scanned by the count pass's last
    // CTA (one launch fewer on the chain); larger frames take the scan kernel
    // (with stage events on, the count and scan launches stay apart)
    const unsigned heavy_epoch = ++h->heavy_epoch, scan_epoch = ++h->scan_epoch;
    const bool fused = !ev && launch_count_and_scan(h->g, T, s->tris, V, h->vtx, h->rect, h->bin_count, h->status,
                                                    h->stats, h->num_sms, st, clip_tris, clip_cap, h->exact_bins,
                                                    h->heavy, heavy_cap(h), heavy_epoch, h->bin_off, h->cursor,
                                                    (unsigned long long)h->ecap, h->chunk_state, scan_epoch);
    if (!fused) {
      launch_setup_count(h->g, T, s->tris, V, h->vtx, h->rect, h->bin_count, h->status, h->stats, h->num_sms, st,
                         clip_tris, clip_cap, h->exact_bins, h->heavy, heavy_cap(h), heavy_epoch);
      if (ev) cudaEventRecord(h->stage_ev[2], st);
      launch_scan(h->nbins, h->bin_count, h->bin_off, h->cursor, (unsigned long long)h->ecap, h->status,
                  h->chunk_state, scan_epoch, st, h->wait_budget, h->withhold);
      if (ev) cudaEventRecord(h->stage_ev[3], st);
    }
    if (!h->check_capacity) break;
    cudaError_t e = cudaMemcpyAsync(h->h_needed, &h->status->needed, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "bin-list size read-back");
    const long long need = (long long)*h->h_needed;
    if (need <= h->ecap) break;
    if (attempt > 0 || need > 0xFFFFFFF0LL) return fail(h, PIKO_ERR_OVERFLOW, "bin lists too large");
    if ((r = grow(h, &h->bin_tris, &h->ecap, need, "bin lists")) != PIKO_OK) return r;
    // the failed scan recorded an overflow and zeroed the counts: clear and count again
    e = cudaMemsetAsync(h->status, 0, sizeof(unsigned) * 2, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "status clear");
  }
  launch_scatter(h->g, T, h->rect, h->bin_off, h->cursor, h->bin_tris, (unsigned long long)h->ecap, h->status,
                 h->num_sms, st, clip_tris, clip_cap, h->exact_bins ? s->tris : nullptr, V, h->vtx, h->heavy,
                 heavy_cap(h), h->heavy_epoch);
  if (ev) cudaEventRecord(h->stage_ev[4], st);

  ProcessParams p;
  p.g = h->g;
  p.ntiles = h->nbins;
  // records sized from this frame's bin-list total when it was read back,
  // else from the last one read back
  if (h->check_capacity) h->last_entries = (long long)*h->h_needed;
  p.slots_hint = slots_for_entries(h->last_entries, h->nbins);
  p.schedule = h->schedule;
  p.small_px = h->small_px;
  p.mode = s->shade_mode;
  p.unclamped = h->unclamped;
  p.stats = h->stats;
  p.num_triangles = T;
  p.tris = s->tris;
  p.vtx = h->vtx;
  p.color = s->color;
  p.normal = s->normal;
  p.light = s->light_dir;
  p.vdot = h->vdot;
  p.invw = h->perspective ? h->invw : nullptr;
  p.clip_tris = clip_tris;
  p.clip_orig = h->clip ? h->clip_orig : nullptr;
  p.pos = s->pos;
  p.mvp = s->mvp;
  p.bin_off = h->bin_off;
  p.bin_tris = h->bin_tris;
  p.key_out = reinterpret_cast<unsigned long long*>(fb->key);
  p.rgba_out = reinterpret_cast<float4*>(fb->rgba);
  p.gnorm_out = reinterpret_cast<uint2*>(fb->gbuf_normal);
  p.galb_out = reinterpret_cast<uint2*>(fb->gbuf_albedo);
  p.st = h->status;
  int grid = h->nbins;
  if (h->schedule != PIKO_SCHED_HARDWARE) {
    int per_sm = 0;
    cudaError_t e = process_occupancy(p, h->threads, &per_sm);
    if (e != cudaSuccess) return cuda_fail(h, e, "occupancy query");
    if (per_sm < 1) per_sm = 1;
    grid = per_sm * h->num_sms < h->nbins ? per_sm * h->num_sms : h->nbins;
  }
  cudaError_t e = launch_process(p, h->threads, grid, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "process launch");
  if (ev) cudaEventRecord(h->stage_ev[5], st);
  return PIKO_OK;
}

int piko_raster_forward_host(piko_raster* h, const piko_scene* s, piko_framebuffer* fb, void* cuda_stream) {
  if (!h || !s || !fb) return PIKO_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (s->width != h->W || s->height != h->H) return fail(h, PIKO_ERR_INVALID_ARG, "scene size differs from the handle's");
  if (s->num_vertices < 0 || s->num_triangles < 0) return fail(h, PIKO_ERR_INVALID_ARG, "negative counts");
  if ((s->num_vertices > 0 && !s->pos) || (s->num_triangles > 0 && !s->tris) || !fb->key)
    return fail(h, PIKO_ERR_INVALID_ARG, "NULL required pointer");
  const long long V = s->num_vertices, T = s->num_triangles, P = (long long)h->W * h->H;
  const bool gbuf = s->shade_mode == PIKO_SHADE_GBUFFER;
  // device buffers (grown on first use; a growth synchronizes the device)
  int r = PIKO_OK;
  if (r == PIKO_OK) r = grow(h, &h->hs_pos, &h->hcap_pos, V, "host-scene positions");
  if (r == PIKO_OK) r = grow(h, &h->hs_tris, &h->hcap_tris, 3 * T, "host-scene triangles");
  if (r == PIKO_OK && s->color) r = grow(h, &h->hs_color, &h->hcap_color, 3 * V, "host-scene colours");
  if (r == PIKO_OK && s->normal) r = grow(h, &h->hs_normal, &h->hcap_normal, 3 * V, "host-scene normals");
  if (r == PIKO_OK) r = grow(h, &h->hs_small, &h->hcap_small, 20, "host-scene matrix and light");
  if (r == PIKO_OK) r = grow(h, &h->hs_key, &h->hcap_key, P, "host-framebuffer keys");
  if (r == PIKO_OK && fb->rgba && !gbuf) r = grow(h, &h->hs_rgba, &h->hcap_rgba, P, "host-framebuffer colour");
  if (r == PIKO_OK && gbuf && fb->gbuf_normal) r = grow(h, &h->hs_gn, &h->hcap_gn, P, "host G-buffer normals");
  if (r == PIKO_OK && gbuf && fb->gbuf_albedo) r = grow(h, &h->hs_ga, &h->hcap_ga, P, "host G-buffer albedo");
  if (r != PIKO_OK) return r;
  piko_scene ds = *s;
  ds.pos = reinterpret_cast<const float*>(h->hs_pos);
  ds.tris = h->hs_tris;
  ds.color = s->color ? h->hs_color : nullptr;
  ds.normal = s->normal ? h->hs_normal : nullptr;
  ds.mvp = s->mvp ? h->hs_small : nullptr;
  ds.light_dir = s->light_dir ? h->hs_small + 16 : nullptr;
  r = check_scene(h, &ds);  // every argument check before anything is enqueued
  if (r != PIKO_OK) return r;
  piko_framebuffer dfb = {};
  struct Copy {
    void* dst;
    const void* src;
    size_t bytes;
  };
  const Copy in[] = {
      {h->hs_pos, s->pos, (size_t)V * 16},
      {h->hs_tris, s->tris, (size_t)T * 12},
      {h->hs_color, s->color, s->color ? (size_t)V * 12 : 0},
      {h->hs_normal, s->normal, s->normal ? (size_t)V * 12 : 0},
      {h->hs_small, s->mvp, s->mvp ? (size_t)64 : 0},
      {h->hs_small + 16, s->light_dir, s->light_dir ? (size_t)12 : 0},
  };
  for (const Copy& c : in) {
    if (c.bytes == 0) continue;
    const cudaError_t e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "host-to-device copy");
  }
  dfb.key = reinterpret_cast<uint64_t*>(h->hs_key);
  dfb.rgba = fb->rgba && !gbuf ? reinterpret_cast<float*>(h->hs_rgba) : nullptr;
  dfb.gbuf_normal = gbuf && fb->gbuf_normal ? h->hs_gn : nullptr;
  dfb.gbuf_albedo = gbuf && fb->gbuf_albedo ? h->hs_ga : nullptr;
  r = piko_raster_forward(h, &ds, &dfb, cuda_stream);
  if (r != PIKO_OK) return r;
  const Copy out[] = {
      {fb->key, dfb.key, (size_t)P * 8},
      {fb->rgba, dfb.rgba, dfb.rgba ? (size_t)P * 16 : 0},
      {fb->gbuf_normal, dfb.gbuf_normal, dfb.gbuf_normal ? (size_t)P * 8 : 0},
      {fb->gbuf_albedo, dfb.gbuf_albedo, dfb.gbuf_albedo ? (size_t)P * 8 : 0},
  };
  for (const Copy& c : out) {
    if (c.bytes == 0) continue;
    const cudaError_t e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "device-to-host copy");
  }
  return PIKO_OK;
}

int piko_raster_forward_batch(piko_raster* h, const piko_scene* scenes, int n, piko_framebuffer* fbs,
                              const int32_t* bin_sizes, const int32_t* schedules, void* cuda_stream) {
  if (!h) return PIKO_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->last_stream = st;
  if (h->clip) return fail(h, PIKO_ERR_INVALID_ARG, "near/far clipping is available for single scenes only");
  // the batch deals tiles inside one launch: the other mappings fall back to its dynamic schedule
  const int dsched = h->schedule > PIKO_SCHED_HARDWARE ? PIKO_SCHED_DYNAMIC : h->schedule;
  int r = batch_prepare(h->batch, h->num_sms, scenes, n, fbs, bin_sizes, schedules, h->bin_w, h->bin_h, dsched,
                        h->unclamped, h->perspective, st, h->err);
  if (r != PIKO_OK) return r;
  for (int attempt = 0;; ++attempt) {
    if ((r = batch_launch_forward(h->batch, h->status, h->batch_launch == 0, st, h->err, h->wait_budget,
                                  h->withhold)) != PIKO_OK)
      return r;
    if (!h->check_capacity) return PIKO_OK;
    cudaError_t e = cudaMemcpyAsync(h->h_needed, &h->status->needed, sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "batch bin-list size read-back");
    const long long need = (long long)*h->h_needed;
    batch_note_entries(h->batch, need);
    if (need <= batch_capacity(h->batch)) return PIKO_OK;
    if (attempt > 0 || need > 0xFFFFFFF0LL) return fail(h, PIKO_ERR_OVERFLOW, "batch bin lists too large");
    if ((r = batch_grow_entries(h->batch, need, h->err)) != PIKO_OK) return r;
    e = cudaMemsetAsync(h->status, 0, sizeof(unsigned) * 2, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "status clear");
  }
}

int piko_raster_backward_batch(piko_raster* h, const piko_scene* scenes, int n, const piko_framebuffer* fbs,
                               const float* const* dl_drgba, float* const* dl_dcolor, float* const* dl_dnormal,
                               float* const* dl_dlight, void* cuda_stream) {
  if (!h) return PIKO_ERR_INVALID_ARG;
  if (!scenes || !fbs || n < 1) return fail(h, PIKO_ERR_INVALID_ARG, "backward_batch needs scenes and framebuffers");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->last_stream = st;
  return batch_launch_backward(h->batch, scenes, n, fbs, dl_drgba, dl_dcolor, dl_dnormal, dl_dlight, h->num_sms, st,
                               h->err);
}

int piko_raster_set_stage_events(piko_raster* h, void* const* events, int n) {
  if (!h) return PIKO_ERR_INVALID_ARG;
  if (n == 0 && !events) {
    h->use_stage_ev = false;
    return PIKO_OK;
  }
  if (n != PIKO_NUM_STAGE_EVENTS || !events) return fail(h, PIKO_ERR_INVALID_ARG, "need PIKO_NUM_STAGE_EVENTS events");
  for (int i = 0; i < n; ++i) {
    if (!events[i]) return fail(h, PIKO_ERR_INVALID_ARG, "NULL event");
    h->stage_ev[i] = reinterpret_cast<cudaEvent_t>(events[i]);
  }
  h->use_stage_ev = true;
  return PIKO_OK;
}

int piko_raster_stats(piko_raster* h, int64_t out[5]) {
  if (!h || !out) return PIKO_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(h->last_stream);
  DevStatus st;
  if (e == cudaSuccess) e = cudaMemcpy(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "stats read");
  out[0] = (int64_t)st.needed;
  out[1] = (int64_t)st.tests;
  out[2] = (int64_t)st.frags;
  out[3] = (int64_t)st.shaded;
  out[4] = (int64_t)st.binned;
  return PIKO_OK;
}

int piko_raster_backward(piko_raster* h, const piko_scene* s, const piko_framebuffer* fwd, const float* dl_drgba,
                         float* dl_dcolor, float* dl_dnormal, float* dl_dlight, void* cuda_stream) {
  if (!h) return PIKO_ERR_INVALID_ARG;
  int r = check_scene(h, s);
  if (r != PIKO_OK) return r;
  if (s->shade_mode == PIKO_SHADE_GBUFFER)
    return fail(h, PIKO_ERR_INVALID_ARG, "backward is defined for Gouraud and Lambert shading");
  if (!fwd || !fwd->key || !dl_drgba) return fail(h, PIKO_ERR_INVALID_ARG, "backward needs the forward key and dL/drgba");
  if (!aligned16(dl_drgba)) return fail(h, PIKO_ERR_INVALID_ARG, "dl_drgba must be 16-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->last_stream = st;
  if ((r = grow(h, &h->vtx, &h->vcap, s->num_vertices, "vertex buffer")) != PIKO_OK) return r;
  if (h->perspective && (r = grow(h, &h->invw, &h->icap, s->num_vertices, "vertex 1/w")) != PIKO_OK) return r;
  float* invw = h->perspective ? h->invw : nullptr;
  // the vertex stage runs again so that backward does not depend on which
  // scene the handle rasterized last
  launch_vertex(h->W, h->H, s->num_vertices, s->pos, s->mvp, h->vtx, nullptr, nullptr, nullptr, invw, h->num_sms,
                st);
  if (piko_backward_launch(h->W, h->H, s->shade_mode, h->unclamped, s->num_triangles, s->num_vertices, s->tris,
                           h->vtx, s->color, s->normal, s->light_dir, invw, h->clip ? s->pos : nullptr, s->mvp,
                           reinterpret_cast<const unsigned long long*>(fwd->key), dl_drgba, dl_dcolor,
                           dl_dnormal, dl_dlight, h->num_sms, st) != 0)
    return cuda_fail(h, cudaGetLastError(), "backward launch");
  return PIKO_OK;
}

int piko_raster_deferred_light(piko_raster* h, const piko_framebuffer* gbuf, const float* lights, int n_lights,
                               float* rgba_out, void* cuda_stream) {
  if (!h) return PIKO_ERR_INVALID_ARG;
  if (!gbuf || !gbuf->key || !gbuf->gbuf_normal || !gbuf->gbuf_albedo || !rgba_out || !lights)
    return fail(h, PIKO_ERR_INVALID_ARG, "deferred light needs key, G-buffer, lights and output");
  if (n_lights < 1 || n_lights > 1024) return fail(h, PIKO_ERR_INVALID_ARG, "n_lights must be in 1..1024");
  if (!aligned16(lights) || !aligned16(rgba_out) || !aligned16(gbuf->gbuf_normal) || !aligned16(gbuf->gbuf_albedo))
    return fail(h, PIKO_ERR_INVALID_ARG, "lights, G-buffer and output must be 16-byte aligned");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  h->last_stream = st;
  launch_deferred_light(h->W, h->H, reinterpret_cast<const unsigned long long*>(gbuf->key), reinterpret_cast<const uint2*>(gbuf->gbuf_normal),
                        reinterpret_cast<const uint2*>(gbuf->gbuf_albedo), reinterpret_cast<const float4*>(lights),
                        n_lights, reinterpret_cast<float4*>(rgba_out), h->num_sms, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PIKO_OK : cuda_fail(h, e, "deferred light launch");
}

}  // extern "C"
