/*
 * piko_raster.h -- C ABI of the GB300 binned forward rasterizer.
 *
 * The library implements the spatially binned raster pipeline of
 * "Piko: A Design Framework for Programmable Graphics Pipelines" (Patney et
 * al., arXiv 1404.6293) as fixed CUDA kernels for sm_103a: a vertex stage,
 * fixed-point triangle setup, AssignBin into screen tiles (count, scan,
 * scatter), a Schedule of tiles onto CTAs, and a per-tile Process stage that
 * resolves coverage, depth and shading.  Sec. 4.1 of the paper (Table of
 * phases: AssignBin per primitive, Schedule per bin, Process per bin) gives
 * the stage structure; Sec. 7.1 names the raster stages (vertex shader,
 * rasterizer, fragment shader, depth test, composite); Listing 1 gives the
 * Lambert fragment shader.
 *
 * Conventions for every call:
 *  - All data pointers are CUDA device pointers owned by the caller, except
 *    where a parameter says host.  The library never frees caller memory.
 *  - Calls enqueue work on the caller's stream (a cudaStream_t passed as
 *    void*, NULL = legacy default stream) and return without waiting, except
 *    where stated.  Host-side argument checks are synchronous.
 *  - Every int-returning call returns a PIKO_* status; on failure
 *    piko_raster_last_error() describes it.  Conditions found on the device
 *    (bad index, bin-list overflow, timeout) are recorded in a device status
 *    word that piko_raster_status() reads.
 *  - A handle owns its scratch memory (vertex and bin buffers) and is not
 *    thread-safe; use one handle per host thread.
 *  - Pixel (x, y) is stored at y*width + x, row 0 at the top of the image.
 *
 * Rasterization rules (the paper is silent on bit-level rules; these are the
 * library's definition, identical to its CPU oracle):
 *  - clip = M * pos in float32, rows summed left to right without fused
 *    multiply-add; a vertex with clip.w <= 0 or NaN, NDC z outside [-1,1],
 *    or a snapped coordinate outside +-2^23 culls its triangles.
 *  - viewport: sx = (x*0.5+0.5)*W, sy = (0.5-y*0.5)*H, sz = (z*0.5+0.5)*(2^24-1);
 *    16.8 fixed point X = rint(256 sx), Y = rint(256 sy), Z = rint(sz).
 *  - int64 edge functions, top-left fill rule, samples at pixel centres;
 *    depth z = floor(sum_i w_i Z_i / A) exactly; the pixel keeps the
 *    minimum of key = (z << 32) | triangle index (nearest wins, ties to the
 *    lower index).  Empty pixels keep key 0xFFFFFFFFFFFFFFFF.
 */
#ifndef PIKO_RASTER_H
#define PIKO_RASTER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define PIKO_OK 0
#define PIKO_ERR_INVALID_ARG 1 /* rejected on the host; nothing was enqueued    */
#define PIKO_ERR_CUDA 2        /* a CUDA call failed; see piko_raster_last_error */
#define PIKO_ERR_OOM 3         /* scratch allocation failed                      */
#define PIKO_ERR_OVERFLOW 4    /* bin lists exceeded the reserved capacity       */
#define PIKO_ERR_TIMEOUT 5     /* a bounded device-side wait gave up             */
#define PIKO_ERR_BAD_INDEX 6   /* a triangle referenced a vertex outside [0, V)  */

/* ---- tile schedules (Sec. 4.3, Schedule directives; Sec. 6) ------------ */
#define PIKO_SCHED_STATIC 0   /* DirectMap: persistent CTA c takes tiles c, c+G, c+2G, ...   */
#define PIKO_SCHED_DYNAMIC 1  /* LoadBalance: persistent CTAs pop tiles from an atomic queue */
#define PIKO_SCHED_HARDWARE 2 /* one CTA per tile, balanced by the hardware block scheduler
                                 (the schedule elimination of Sec. 5.2.2)                   */
/* Two other mappings of the same pipeline, for the design-space comparison of
 * Sec. 7.2 (same keys and colours; bin size and threads per tile unused):   */
#define PIKO_SCHED_FUSED 3    /* full fusion without tiling (the FreePipe-style point of
                                 Sec. 7.2): one pass over the triangles takes a 64-bit
                                 atomic minimum on the key buffer in global memory, then
                                 every pixel is shaded from its winner                     */
#define PIKO_SCHED_UNFUSED 4  /* the Baseline pipeline of Sec. 7.1, one kernel per stage:
                                 rasterizer (every covered sample to a global fragment
                                 buffer), fragment shader (every fragment), depth test,
                                 composite.  The fragment buffer grows like the bin lists
                                 (PIKO_OPT_CHECK_CAPACITY); its overflow is reported as
                                 PIKO_ERR_OVERFLOW.  Batches treat both as DYNAMIC.  Work
                                 counters (piko_raster_stats) are not kept on these two.  */

/* ---- shading modes ---------------------------------------------------- */
#define PIKO_SHADE_GOURAUD 0 /* rgb = sum b_i c_i                                         */
#define PIKO_SHADE_LAMBERT 1 /* rgb = albedo * max(0, n . L): diffuse (Sec. 4.1 example) */
#define PIKO_SHADE_GBUFFER 2 /* no colour; FP16 normal and albedo for a deferred light pass */

/* ---- options for piko_raster_set_option ------------------------------- */
#define PIKO_OPT_THREADS_PER_TILE 1 /* CTA size of the Process stage: 64, 128, 256 or 512
                                       (the threads-per-bin knob of Listing 1 / Sec. 6);
                                       default 64 for bins of at most 64 pixels, 128 up to
                                       256 pixels, 256 above, and 512 when the frame has
                                       fewer bins than twice the GPU's SMs                  */
#define PIKO_OPT_UNCLAMPED 2        /* 1: Lambert without the max(0, .) clamp,
                                       rgb = albedo * (n . L); default 0 (clamped)         */
#define PIKO_OPT_CHECK_CAPACITY 3   /* 1 (default): forward reads the bin-list size back
                                       after the scan (one host sync) and grows scratch
                                       before scattering; 0: no sync, overflow is reported
                                       as PIKO_ERR_OVERFLOW by piko_raster_status          */
#define PIKO_OPT_SCHEDULE 4         /* change the schedule (PIKO_SCHED_*)                   */
#define PIKO_OPT_SMALL_TRI_PIXELS 5 /* triangles whose box inside a tile has at most this
                                       many pixels are rasterized by one thread; larger ones
                                       by a whole warp (default 32)                         */
#define PIKO_OPT_STATS 6            /* 1: the Process stage also counts its work (see
                                       piko_raster_stats); default 0                        */
#define PIKO_OPT_BATCH_LAUNCH 7     /* how piko_raster_forward_batch launches its phases:
                                       0 (default) one persistent cooperative kernel with grid
                                       barriers between phases; 1 one launch per phase     */
#define PIKO_OPT_PERSPECTIVE 8      /* 1: perspective-correct attributes in shading and
                                       gradients: b'_i = (b_i / w_i) / sum_j (b_j / w_j), w_i
                                       the clip w of vertex i; 0 (default): screen-space b_i.
                                       Depth and coverage do not change.  Applies to every
                                       scene of a batch; piko_raster_backward_batch follows
                                       the setting of the last piko_raster_forward_batch,
                                       piko_raster_backward the handle's current setting  */
#define PIKO_OPT_CLIP 11            /* 1: near/far clipping instead of culling: a triangle with
                                       a vertex outside -w <= z <= w (or w not > 0) is clipped
                                       against z = -w, then z = w, in clip space; the polygon
                                       is fanned into sub-triangles that rasterize with the
                                       triangle's index in the key, and a clipped triangle is
                                       shaded (and differentiated) from its vertices with the
                                       clip-space weights of each pixel centre's ray
                                       (perspective-correct).  Single-scene calls only
                                       (piko_raster_forward_batch rejects it); the sub-triangle
                                       list grows like the bin lists.  Default 0: culling      */
#define PIKO_OPT_EXACT_BINS 12      /* 1: AssignBin gives a triangle that spans several bins
                                       an entry only in the bins it overlaps: none of its
                                       three edges may fail the fill-rule test at every
                                       pixel centre of the bin inside its bounding box (the
                                       separating-axis test of the triangle against that
                                       rectangle of centres).  Fewer bin entries for large
                                       and thin triangles, identical output; the count and
                                       scatter passes do the test.  Single-scene calls;
                                       piko_raster_forward_batch bins by bounding box.
                                       Default 0: bounding-box bins (AssignToBoundingBox) */
#define PIKO_OPT_WAIT_BUDGET 9      /* how long a device-side wait (scan look-back, batch grid
                                       barrier) may spin before it gives up, records
                                       PIKO_ERR_TIMEOUT and lets the frame's later phases
                                       skip their work: value x 1000 SM clock cycles,
                                       1..1000000 (default 40000, about 20 ms)              */
#define PIKO_OPT_TEST_WITHHOLD 10   /* test hook for the bounded waits; faults nothing.
                                       Bit 0: scan chunk 0 does not publish its prefix, so
                                       chunk 1's look-back runs out (needs more than 2048
                                       tiles).  Bit 1: in a persistent batch, CTA 0 does not
                                       arrive at the first grid barrier, so every CTA's wait
                                       runs out.  The frame then reports PIKO_ERR_TIMEOUT
                                       and writes no output.  Bit 2: the list of heavy
                                       triangles (spanning 256 bins or more) counts as full,
                                       so their bin entries are written by their own warps;
                                       same output.  Default 0                             */

/* Stage boundaries of one forward pass, for piko_raster_set_stage_events. */
#define PIKO_NUM_STAGE_EVENTS 6 /* before vertex, after vertex, after setup+count, after scan,
                                   after scatter, after process                             */

typedef struct piko_raster piko_raster; /* opaque */

/* A triangle list with per-vertex attributes (the input of the raster
 * pipeline, Sec. 7.1).  All pointers are device memory, caller-owned. */
typedef struct piko_scene {
  int32_t width, height;      /* framebuffer size in pixels, 1..32767          */
  int32_t num_vertices;       /* V >= 0                                         */
  int32_t num_triangles;      /* T >= 0                                         */
  const float *pos;           /* [V][4] homogeneous x,y,z,w; 16-byte aligned    */
  const int32_t *tris;        /* [T][3] vertex indices; 16-byte aligned         */
  const float *color;         /* [V][3] RGB (albedo), or NULL                   */
  const float *normal;        /* [V][3], required by LAMBERT and GBUFFER        */
  const float *mvp;           /* [16] row-major 4x4 applied to pos, NULL = I    */
  const float *light_dir;     /* [3] directional light L, used as given         */
  int32_t shade_mode;         /* PIKO_SHADE_*                                   */
  int32_t reserved;           /* must be 0                                      */
} piko_scene;

/* Caller-owned device outputs of a forward pass. */
typedef struct piko_framebuffer {
  uint64_t *key;     /* [H][W] (depth << 32) | triangle index; required              */
  float *rgba;       /* [H][W][4] shaded colour, alpha 1 where covered; NULL allowed */
  void *gbuf_normal; /* [H][W][4] binary16 (nx, ny, nz, 0), GBUFFER mode only        */
  void *gbuf_albedo; /* [H][W][4] binary16 (r, g, b, 1),   GBUFFER mode only        */
} piko_framebuffer;

/* Creates a rasterizer for width x height framebuffers with bin_w x bin_h
 * pixel tiles (each in {8, 16, 32, 64}; Sec. 3 and the bin-size template
 * parameters of Listing 1) and a PIKO_SCHED_* tile schedule.  Returns NULL
 * on invalid arguments (width or height outside 1..32767) or if CUDA fails.
 * Allocates a little device memory on the current device; larger scratch
 * is allocated on first use or by piko_raster_reserve. */
piko_raster *piko_raster_create(int width, int height, int bin_w, int bin_h, int schedule);

/* Frees the handle's scratch memory (synchronizes the device first). */
void piko_raster_destroy(piko_raster *h);

/* Forward pass (Sec. 7.1 stages; AssignBin/Schedule/Process of Sec. 4.1):
 * vertex stage -> triangle setup and per-bin counts -> scan -> scatter of
 * triangle indices into bin lists -> per-tile coverage, depth and shading.
 * scene->width/height must equal the handle's.  Writes every pixel of
 * fb->key and of fb->rgba (if not NULL; zero where empty) or, in GBUFFER
 * mode, of fb->gbuf_normal and fb->gbuf_albedo.  Asynchronous unless
 * PIKO_OPT_CHECK_CAPACITY is 1 (the default), which adds one host sync
 * after the scan.  Returns PIKO_ERR_INVALID_ARG for bad sizes, NULL
 * required pointers, misaligned pos/tris, or a shade mode without the
 * attributes it needs.  The stages after the vertex stage are launched with
 * programmatic dependent launch: each may start while the one before it
 * drains and waits on the device before reading that stage's output. */
int piko_raster_forward(piko_raster *h, const piko_scene *scene, piko_framebuffer *fb,
                        void *cuda_stream);

/* The forward pass of a scene held in HOST memory into a framebuffer in host
 * memory (the paper's problem statement end to end: a triangle list with
 * per-vertex attributes in, a framebuffer out, Sec. 7.1).  scene and fb are
 * as for piko_raster_forward except that every array pointer (pos, tris,
 * color, normal, mvp, light_dir; key, rgba, gbuf_normal, gbuf_albedo) is
 * host memory, with no alignment requirement; page-locked memory
 * (cudaHostAlloc, or pinned tensors) makes the copies asynchronous.  The
 * handle copies the arrays into device buffers it owns (allocated on first
 * use and grown when a larger scene or framebuffer comes, which
 * synchronizes the device), runs piko_raster_forward on them and copies
 * fb's requested outputs back, all enqueued on cuda_stream in that order;
 * the caller must not touch the host arrays until the stream has passed
 * this call.  Errors: PIKO_ERR_INVALID_ARG (size differs from the handle's,
 * negative counts, a NULL required pointer, a shade mode without the
 * attributes it needs; nothing enqueued), PIKO_ERR_OOM (a device buffer
 * could not grow; nothing enqueued), the codes of piko_raster_forward, and
 * PIKO_ERR_CUDA for a failed copy. */
int piko_raster_forward_host(piko_raster *h, const piko_scene *scene, piko_framebuffer *fb,
                             void *cuda_stream);

/* Gradients of a loss through shading with visibility held fixed by a
 * previous forward's fwd->key (the coverage stays exact integer
 * arithmetic).  dl_drgba [H][W][4] is dLoss/d(rgba) (alpha ignored).
 * Accumulates (+=) into dl_dcolor [V][3], dl_dnormal [V][3] and dl_dlight
 * [3]; any of them may be NULL to skip it.  GOURAUD: colour only; LAMBERT:
 * colour (if scene->color), normal and light.  The caller zeroes the
 * outputs.  Not defined by the paper; the gradients are those of the
 * shading formulas of Listing 1. */
int piko_raster_backward(piko_raster *h, const piko_scene *scene, const piko_framebuffer *fwd,
                         const float *dl_drgba, float *dl_dcolor, float *dl_dnormal,
                         float *dl_dlight, void *cuda_stream);

/* Deferred light pass over a G-buffer written by a GBUFFER forward: for each
 * covered pixel, sum of n_lights point lights (lights: device [n][4] =
 * x, y, z in pixel units, intensity) with
 *   S = (x + 0.5, y + 0.5, depth / (2^24-1) * D),  D = max(W, H), r = D/4,
 *   rgb = albedo * sum_l I_l max(0, n . (P_l - S)/|P_l - S|) / (1 + |P_l - S|^2 / r^2),
 * alpha 1; empty pixels get 0.  Shader complexity as the number of lights is
 * the axis of Fig. (a) of the paper's Sec. 7.2; the light model itself is
 * this library's.  1 <= n_lights <= 1024. */
int piko_raster_deferred_light(piko_raster *h, const piko_framebuffer *gbuf, const float *lights,
                               int n_lights, float *rgba_out, void *cuda_stream);

/* Many scenes in one pass (scenes with uneven triangle counts and
 * resolutions, or many views of one mesh): vertex stage, setup and counts,
 * scan, scatter and Process for all n scenes run as one persistent
 * cooperative launch whose CTAs meet at grid barriers between the phases
 * (PIKO_OPT_BATCH_LAUNCH = 1: one launch per phase instead).  The paper's
 * runtime is multi-kernel (Sec. 5, Sec. 6) and names a persistent kernel as
 * the alternative; scenes, bins and tiles of all scenes share one index
 * space here.
 *  scenes, fbs  host arrays of n descriptors (their pointers are device
 *               memory); each scene has its own width and height
 *               (1..32767) and shading mode, and writes its own framebuffer.
 *  bin_sizes    host int32 [n][2] (bin width, height per scene, each in
 *               {8,16,32,64}), or NULL for the handle's bin size.
 *  schedules    host int32 [n] PIKO_SCHED_STATIC (the scene's tiles are dealt
 *               round robin over the persistent CTAs) or PIKO_SCHED_DYNAMIC
 *               (taken from a shared queue after the static tiles; HARDWARE
 *               is treated as DYNAMIC), or NULL for the handle's schedule.
 * Keys are bit-identical to n piko_raster_forward calls with the same bin
 * sizes; colours agree with them within float32 rounding (a winner is
 * shaded from its tile's shared-memory record or, past the records a tile
 * holds, from global memory).  With PIKO_OPT_CHECK_CAPACITY = 1 the call waits for the
 * launch, and relaunches once with larger bin lists if they overflowed; with
 * 0 it never waits (so it can be captured in a CUDA graph after a first call
 * with the same scenes, or piko_raster_reserve, has sized the scratch) and
 * reports overflow through piko_raster_status.  A grid barrier or scan wait
 * that runs out of its time budget records PIKO_ERR_TIMEOUT and every later
 * phase is skipped.  The batch keeps its own scratch in the handle; n >= 1,
 * sum of vertices and of triangles below 2^31. */
int piko_raster_forward_batch(piko_raster *h, const piko_scene *scenes, int n, piko_framebuffer *fbs,
                              const int32_t *bin_sizes, const int32_t *schedules, void *cuda_stream);

/* Gradients for all scenes of the last piko_raster_forward_batch on this
 * handle (same scenes, same order), in one launch: dl_drgba, dl_dcolor,
 * dl_dnormal and dl_dlight are host arrays of n device pointers (entries
 * may be NULL to skip that output for a scene); semantics per scene as in
 * piko_raster_backward (accumulated, visibility fixed by fbs[i].key). */
int piko_raster_backward_batch(piko_raster *h, const piko_scene *scenes, int n, const piko_framebuffer *fbs,
                               const float *const *dl_drgba, float *const *dl_dcolor, float *const *dl_dnormal,
                               float *const *dl_dlight, void *cuda_stream);

/* Pre-sizes scratch for scenes of up to max_vertices / max_triangles and
 * max_bin_entries (triangle, tile) pairs, so that later forwards allocate
 * nothing (required before capturing forwards in a CUDA graph).
 * Synchronous. */
int piko_raster_reserve(piko_raster *h, int64_t max_vertices, int64_t max_triangles,
                        int64_t max_bin_entries);

/* Sets a PIKO_OPT_* option.  Returns PIKO_ERR_INVALID_ARG for unknown keys
 * or values. */
int piko_raster_set_option(piko_raster *h, int key, int value);

/* Waits for the handle's last stream, returns the device status word
 * (PIKO_OK or the first PIKO_ERR_* recorded since the last call) and clears
 * it.  If needed_bin_entries is not NULL it receives the bin-list size the
 * last scan required. */
int piko_raster_status(piko_raster *h, int64_t *needed_bin_entries);

/* Makes the next piko_raster_forward record the PIKO_NUM_STAGE_EVENTS
 * caller-created CUDA events (cudaEvent_t passed as void*) on its stream at
 * the stage boundaries listed above, for per-stage timing without extra
 * synchronisation.  The events are used by that one forward only.  n must
 * be PIKO_NUM_STAGE_EVENTS, or 0 with events NULL to cancel. */
int piko_raster_set_stage_events(piko_raster *h, void *const *events, int n);

/* Work counted by the last forward run with PIKO_OPT_STATS = 1 (waits for
 * the stream): out[0] bin entries, out[1] pixel samples tested (pixels of
 * each triangle's bounding box inside each of its tiles), out[2] covered
 * samples (rasterized fragments, occluded ones included), out[3] covered
 * pixels after the depth test (shaded fragments), out[4] triangles that
 * survived culling and reached a bin. */
int piko_raster_stats(piko_raster *h, int64_t out[5]);

/* ---- forward pass without any device allocation ------------------------
 * The paper has no counterpart; this entry point exists for callers that
 * are not allowed to allocate GPU memory: work recorded inside a CUDA stream
 * capture that must not add allocations, plugins whose host application
 * owns the device allocator, and real-time loops that cannot afford the
 * implicit synchronisation of cudaMalloc/cudaFree.
 *
 * It computes what piko_raster_forward computes with the same bin size and
 * schedule and the default options, but needs no handle: its scratch memory
 * is one fixed device array of about 6.3 MB inside this library, which every
 * GPU that loads the library keeps until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.  Its Process launch
 * sizes the per-tile shading records for the largest count the key layout
 * allows (the handle forward sizes them from the last frame's bin lists), so
 * its shared-memory footprint can differ; the output is the same.
 *  - The first call in each CUDA context (for callers on the runtime's
 *    primary context: once per device, with that device current) looks up
 *    the array's device address; make that first call before any stream
 *    capture.  A thread with no current context uses the current device's
 *    primary context.
 *  - Every call on a device shares the array and it keeps the previous
 *    call's contents (each call clears the status word, the scan states and
 *    the per-tile counts itself).  Calls whose work overlaps on the GPU --
 *    on different streams or from different host threads -- race and give
 *    wrong results; order them on one stream.
 *  - Scenes above the limits below, or more tiles than
 *    PIKO_NOALLOC_MAX_BINS, are rejected with PIKO_ERR_INVALID_ARG.  When
 *    a host-side argument check fails nothing is enqueued; the other
 *    host-side checks are those of piko_raster_forward.  A CUDA error while
 *    enqueuing returns PIKO_ERR_CUDA, possibly after part of the work was
 *    enqueued.
 *  - status_out (a device int32, may be NULL) receives PIKO_OK or the first
 *    device-side condition when the pass finishes: PIKO_ERR_OVERFLOW if the
 *    bin lists need more than PIKO_NOALLOC_MAX_BIN_ENTRIES entries (the
 *    framebuffer is then not written), PIKO_ERR_BAD_INDEX for an index
 *    outside [0, V) (that triangle is culled). */
#define PIKO_NOALLOC_MAX_VERTICES 65536
#define PIKO_NOALLOC_MAX_TRIANGLES 65536
#define PIKO_NOALLOC_MAX_BINS 16384
#define PIKO_NOALLOC_MAX_BIN_ENTRIES 1048576
int piko_raster_forward_noalloc(const piko_scene *scene, piko_framebuffer *fb, int bin_w, int bin_h,
                                int schedule, int32_t *status_out, void *cuda_stream);

/* Message for the last failing call on this handle (never NULL). */
const char *piko_raster_last_error(const piko_raster *h);

/* Library version as major*10000 + minor*100 + patch. */
int piko_raster_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PIKO_RASTER_H */
