/*
 * piko_oracle.c -- plain CPU oracle of the binned forward rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the timed
 * CPU baseline of the benchmark may load this file's library.  It shares no
 * code with the CUDA path and never calls it.
 *
 * What it computes.  The stages of the paper's Baseline raster pipeline
 * (Sec. 7.1: Vertex Shader -> Rasterizer -> Fragment Shader -> Depth Test ->
 * Composite) for opaque triangles, written as the definitions below, one
 * pixel and one triangle at a time, in fixed order:
 *
 *   O1  clip = M * p with float32 operations, each rounded to nearest, no
 *       fused multiply-add, row r summed as ((m0*x + m1*y) + m2*z) + m3*w.
 *       M absent: clip = p.
 *   O2  a triangle with a vertex whose clip w is not > 0 (NaN included) is
 *       culled; ndc = clip.xyz / clip.w (float32 division).
 *   O3  a triangle with a vertex whose ndc z is outside [-1, 1] is culled
 *       (no near/far clipping).
 *   O4  viewport, row 0 at the top:  sx = (ndc.x*0.5 + 0.5)*W,
 *       sy = (0.5 - ndc.y*0.5)*H,  sz = (ndc.z*0.5 + 0.5)*16777215.
 *   O5  16.8 fixed point: X = rint(sx*256), Y = rint(sy*256) (ties to even),
 *       Z = rint(sz) in [0, 2^24-1]; the triangle is culled unless
 *       |sx*256| < 2^23 and |sy*256| < 2^23 for all its vertices.
 *   O6  A = (X1-X0)(Y2-Y0) - (X2-X0)(Y1-Y0) in int64; A == 0 culls; A < 0
 *       swaps vertices 1 and 2 (their attributes follow) and negates A.
 *   O7  edge a->b: E_ab(P) = (Xb-Xa)(Py-Ya) - (Yb-Ya)(Px-Xa);
 *       w0 = E_12, w1 = E_20, w2 = E_01 (so w0 = A at vertex 0).  An edge is
 *       top-left iff dy < 0, or dy == 0 and dx > 0.  P is covered iff every
 *       w_i > 0, or w_i == 0 on a top-left edge.
 *   O8  samples at pixel centres P = (256*px + 128, 256*py + 128).
 *   O9  depth z = floor((w0*Z0 + w1*Z1 + w2*Z2) / A), exact (128-bit).
 *   O10 key = (z << 32) | triangle index; the pixel keeps the minimum key
 *       over all triangles covering it (nearest depth, ties to the lower
 *       index); an empty pixel keeps 0xFFFFFFFFFFFFFFFF.
 *   O11 shading of the winning triangle in float64 with b_i = w_i / A:
 *       Gouraud rgb = sum b_i c_i; Lambert (the diffuse shader of the paper's
 *       example fragment-shader stage, Sec. 4.1)
 *       rgb = albedo * max(0, n . L) with n = sum b_i n_i (not renormalised)
 *       and albedo = sum b_i c_i, or the constant (0.80, 0.75, 0.65) when no
 *       colours are given.  Covered pixels get alpha 1, empty ones 0.
 *   O12 G-buffer: the interpolated normal and albedo rounded to IEEE binary16
 *       (round to nearest even); a light pass sums 64 point lights per pixel
 *       (light_pass below).
 *   O13 gradients of sum (rgb - target)^2 with visibility fixed.
 *   O14 a triangle with an index outside [0, V) is culled and reported.
 *   O15 optional perspective-correct attributes (flag bit 1 of shade,
 *       backward and loss): the screen-space b_i of O11 are replaced by
 *       b'_i = (b_i / w_i) / sum_j (b_j / w_j), w_i the clip w of vertex i
 *       from O1 (float32, read exactly as a double).  An attribute linear
 *       in the triangle's clip-space (or world-space) plane is then the value
 *       at the point the sample's ray meets the plane, the standard
 *       hyperbolic interpolation; with equal w it reduces to O11.
 *   O16 optional near/far clipping (oracle_set_clipping(1)) in place of the
 *       culls of O2/O3: a triangle with a vertex outside -w <= z <= w (or
 *       with w not > 0) is clipped in clip space, first against z + w >= 0,
 *       then against w - z >= 0 (Sutherland-Hodgman over the edges in
 *       order from vertex 0; a crossing at t = d_a / (d_a - d_b), the new
 *       point a + t (b - a) per component, all float32, each operation
 *       rounded, no fused multiply-add).  The polygon (3 to 5 points) is
 *       fanned from its first point into (p0, p_k, p_k+1).  Each point is
 *       divided, mapped and snapped as in O4/O5, its Z clamped to
 *       [0, 2^24-1] instead of culled, w not > 0 culling its sub-triangle.
 *       Sub-triangles rasterize as in O6-O10 with the original triangle's
 *       index in the key.  A clipped triangle is shaded (and differentiated)
 *       from its original vertices with clip-space weights b = n / sum(n),
 *       n = a x c, a_i = X_i - x W_i, c_i = Y_i - y W_i for the pixel
 *       centre's NDC (x, y): the point where the centre's ray meets the
 *       triangle's plane, i.e. perspective-correct whatever O15's flag.
 *
 * The paper fixes none of the bit-level rules above (fixed-point format,
 * fill rule, depth format, rounding, tie-break, light model); they are the
 * readings this library is defined by.  Parity of those conventions against
 * the paper itself is therefore unpinned; the tests pin this code against
 * closed forms, invariants and an independently written scanline rasterizer.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 *        (no contraction: the vertex stage is defined by separately rounded
 *        float32 operations).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_BAD_INDEX 6
#define KEY_EMPTY 0xFFFFFFFFFFFFFFFFull

typedef unsigned __int128 u128;
typedef __int128 i128;

/* ------------------------------------------------------------------ O1-O5 */
typedef struct {
  int32_t X, Y;
  uint32_t Z;
  int32_t ok;
  double w;      /* clip w (O1), for O15 */
  float c[4];    /* clip coordinates (O1), for O16 */
} ovtx;

/* O16 near/far clipping instead of culling (off by default) */
static int g_clip = 0;
void oracle_set_clipping(int on) { g_clip = on ? 1 : 0; }
int oracle_get_clipping(void) { return g_clip; }

static void vertex_stage_one(int W, int H, const float *p, const float *M, ovtx *o) {
  float c[4];
  if (M) {
    for (int r = 0; r < 4; ++r) {
      float acc = M[4 * r + 0] * p[0];
      acc = acc + M[4 * r + 1] * p[1];
      acc = acc + M[4 * r + 2] * p[2];
      acc = acc + M[4 * r + 3] * p[3];
      c[r] = acc;
    }
  } else {
    c[0] = p[0]; c[1] = p[1]; c[2] = p[2]; c[3] = p[3];
  }
  o->X = 0; o->Y = 0; o->Z = 0; o->ok = 0;
  o->w = (double)c[3];
  for (int k = 0; k < 4; ++k) o->c[k] = c[k];
  if (!(c[3] > 0.0f)) return;                                   /* O2 */
  float nx = c[0] / c[3], ny = c[1] / c[3], nz = c[2] / c[3];
  if (!(nz >= -1.0f && nz <= 1.0f)) return;                     /* O3 */
  float sx = (nx * 0.5f + 0.5f) * (float)W;                     /* O4 */
  float sy = (0.5f - ny * 0.5f) * (float)H;
  float sz = (nz * 0.5f + 0.5f) * 16777215.0f;
  float fx = sx * 256.0f, fy = sy * 256.0f;                     /* O5 */
  if (!(fabsf(fx) < 8388608.0f && fabsf(fy) < 8388608.0f)) return;
  o->X = (int32_t)rintf(fx);
  o->Y = (int32_t)rintf(fy);
  o->Z = (uint32_t)rintf(sz);
  o->ok = 1;
}

static ovtx *vertex_stage_all(int W, int H, int V, const float *pos, const float *M) {
  ovtx *v = (ovtx *)malloc(sizeof(ovtx) * (size_t)(V > 0 ? V : 1));
  for (int i = 0; i < V; ++i) vertex_stage_one(W, H, pos + 4 * (size_t)i, M, &v[i]);
  return v;
}

int oracle_vertex_stage(int W, int H, int V, const float *pos, const float *M,
                        int32_t *X, int32_t *Y, uint32_t *Z, int32_t *ok) {
  for (int i = 0; i < V; ++i) {
    ovtx o;
    vertex_stage_one(W, H, pos + 4 * (size_t)i, M, &o);
    X[i] = o.X; Y[i] = o.Y; Z[i] = o.Z; ok[i] = o.ok;
  }
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ O6-O7 */
typedef struct {
  int64_t X[3], Y[3];
  int64_t Z[3];
  int32_t vid[3]; /* original vertex index in each slot */
  int64_t A;
} otri;

/* returns 1 if the triangle survives culling; sets *bad on an index error */
static int setup_triangle(const ovtx *vs, int V, const int32_t *idx, otri *t, int *bad) {
  for (int k = 0; k < 3; ++k)
    if (idx[k] < 0 || idx[k] >= V) { *bad = 1; return 0; }
  for (int k = 0; k < 3; ++k) {
    const ovtx *o = &vs[idx[k]];
    if (!o->ok) return 0;
    t->X[k] = o->X; t->Y[k] = o->Y; t->Z[k] = o->Z; t->vid[k] = idx[k];
  }
  int64_t A = (t->X[1] - t->X[0]) * (t->Y[2] - t->Y[0]) - (t->X[2] - t->X[0]) * (t->Y[1] - t->Y[0]);
  if (A == 0) return 0;
  if (A < 0) {
    int64_t s;
    int32_t si;
    s = t->X[1]; t->X[1] = t->X[2]; t->X[2] = s;
    s = t->Y[1]; t->Y[1] = t->Y[2]; t->Y[2] = s;
    s = t->Z[1]; t->Z[1] = t->Z[2]; t->Z[2] = s;
    si = t->vid[1]; t->vid[1] = t->vid[2]; t->vid[2] = si;
    A = -A;
  }
  t->A = A;
  return 1;
}

static int64_t edge_fn(const otri *t, int a, int b, int64_t Px, int64_t Py) {
  return (t->X[b] - t->X[a]) * (Py - t->Y[a]) - (t->Y[b] - t->Y[a]) * (Px - t->X[a]);
}

static int top_left(const otri *t, int a, int b) {
  int64_t dx = t->X[b] - t->X[a], dy = t->Y[b] - t->Y[a];
  return dy < 0 || (dy == 0 && dx > 0);
}

/* O7-O9: 1 if pixel (px,py) is covered; then *z holds its depth and w[] the
 * edge functions */
static int cover_and_depth(const otri *t, int px, int py, uint32_t *z, int64_t w[3]) {
  int64_t Px = 256 * (int64_t)px + 128, Py = 256 * (int64_t)py + 128;
  w[0] = edge_fn(t, 1, 2, Px, Py);
  w[1] = edge_fn(t, 2, 0, Px, Py);
  w[2] = edge_fn(t, 0, 1, Px, Py);
  const int tl[3] = {top_left(t, 1, 2), top_left(t, 2, 0), top_left(t, 0, 1)};
  for (int i = 0; i < 3; ++i)
    if (!(w[i] > 0 || (w[i] == 0 && tl[i]))) return 0;
  u128 num = (u128)(uint64_t)w[0] * (u128)(uint64_t)t->Z[0] +
             (u128)(uint64_t)w[1] * (u128)(uint64_t)t->Z[1] +
             (u128)(uint64_t)w[2] * (u128)(uint64_t)t->Z[2];
  *z = (uint32_t)(num / (u128)(uint64_t)t->A);
  return 1;
}

/* ------------------------------------------------------------------ O16 */
typedef struct {
  float c[4];
} cvert;

/* one Sutherland-Hodgman pass: plane 0 keeps z + w >= 0, plane 1 w - z >= 0 */
static int clip_plane(const cvert *in, int n, cvert *out, int plane) {
  int m = 0;
  for (int k = 0; k < n; ++k) {
    const cvert *a = &in[k], *b = &in[(k + 1) % n];
    float da = plane == 0 ? a->c[2] + a->c[3] : a->c[3] - a->c[2];
    float db = plane == 0 ? b->c[2] + b->c[3] : b->c[3] - b->c[2];
    int ina = da >= 0.0f, inb = db >= 0.0f;
    if (ina) out[m++] = *a;
    if (ina != inb) {
      float den = da - db;
      float t = da / den;
      cvert v;
      for (int q = 0; q < 4; ++q) {
        float d = b->c[q] - a->c[q];
        float u = t * d;
        v.c[q] = a->c[q] + u;
      }
      out[m++] = v;
    }
  }
  return m;
}

/* O4/O5 for a clipped point: 1 if it snaps inside the guard band */
static int snap_point(int W, int H, const float *c, int64_t *X, int64_t *Y, int64_t *Z) {
  if (!(c[3] > 0.0f)) return 0;
  float nx = c[0] / c[3], ny = c[1] / c[3], nz = c[2] / c[3];
  float sx = (nx * 0.5f + 0.5f) * (float)W;
  float sy = (0.5f - ny * 0.5f) * (float)H;
  float sz = (nz * 0.5f + 0.5f) * 16777215.0f;
  float fx = sx * 256.0f, fy = sy * 256.0f;
  if (!(fabsf(fx) < 8388608.0f && fabsf(fy) < 8388608.0f)) return 0;
  float zr = rintf(sz);
  if (!(zr >= 0.0f)) zr = 0.0f; /* NaN or below the near plane by rounding */
  if (zr > 16777215.0f) zr = 16777215.0f;
  *X = (int64_t)rintf(fx);
  *Y = (int64_t)rintf(fy);
  *Z = (int64_t)zr;
  return 1;
}

/* orientation and area of a triangle given by snapped points (O6) */
static int setup_points(const int64_t *X, const int64_t *Y, const int64_t *Z, otri *t) {
  for (int k = 0; k < 3; ++k) { t->X[k] = X[k]; t->Y[k] = Y[k]; t->Z[k] = Z[k]; t->vid[k] = -1; }
  int64_t A = (t->X[1] - t->X[0]) * (t->Y[2] - t->Y[0]) - (t->X[2] - t->X[0]) * (t->Y[1] - t->Y[0]);
  if (A == 0) return 0;
  if (A < 0) {
    int64_t s;
    s = t->X[1]; t->X[1] = t->X[2]; t->X[2] = s;
    s = t->Y[1]; t->Y[1] = t->Y[2]; t->Y[2] = s;
    s = t->Z[1]; t->Z[1] = t->Z[2]; t->Z[2] = s;
    A = -A;
  }
  t->A = A;
  return 1;
}

/* 1 if clipping applies to triangle idx (O16): its indices are valid and a
 * vertex failed the vertex stage */
static int needs_clip(const ovtx *vs, int V, const int32_t *idx) {
  if (!g_clip) return 0;
  for (int k = 0; k < 3; ++k)
    if (idx[k] < 0 || idx[k] >= V) return 0;
  return !(vs[idx[0]].ok && vs[idx[1]].ok && vs[idx[2]].ok);
}

/* the sub-triangles of a clipped triangle (at most 3), in fan order */
static int clip_triangle(int W, int H, const ovtx *vs, const int32_t *idx, otri *out) {
  cvert p[8], q[8];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 4; ++c) p[k].c[c] = vs[idx[k]].c[c];
  int n = clip_plane(p, 3, q, 0);
  n = clip_plane(q, n, p, 1);
  int m = 0;
  for (int k = 1; k + 1 < n; ++k) {
    int64_t X[3], Y[3], Z[3];
    const cvert *tri[3] = {&p[0], &p[k], &p[k + 1]};
    int ok = 1;
    for (int j = 0; j < 3 && ok; ++j) ok = snap_point(W, H, tri[j]->c, &X[j], &Y[j], &Z[j]);
    if (ok && setup_points(X, Y, Z, &out[m])) ++m;
  }
  return m;
}

/* All triangles set up: the T input triangles first (valid[i] = survives
 * O2-O6), then the sub-triangles of clipped ones (O16); orig[i] is the input
 * index each one keys with.  *total = T + number of sub-triangles. */
typedef struct {
  otri *ts;
  uint8_t *valid;
  int32_t *orig;
  int64_t total;
} oset;

static oset setup_all(int W, int H, const ovtx *vs, int V, int64_t T, const int32_t *tris, int *bad) {
  oset o;
  int64_t cap = T + 16;
  o.ts = (otri *)malloc(sizeof(otri) * (size_t)cap);
  o.valid = (uint8_t *)malloc((size_t)cap);
  o.orig = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
  o.total = T;
  for (int64_t i = 0; i < T; ++i) {
    o.valid[i] = (uint8_t)setup_triangle(vs, V, tris + 3 * i, &o.ts[i], bad);
    o.orig[i] = (int32_t)i;
  }
  for (int64_t i = 0; i < T; ++i) {
    if (!needs_clip(vs, V, tris + 3 * i)) continue;
    otri sub[3];
    int m = clip_triangle(W, H, vs, tris + 3 * i, sub);
    for (int k = 0; k < m; ++k) {
      if (o.total == cap) {
        cap = 2 * cap;
        o.ts = (otri *)realloc(o.ts, sizeof(otri) * (size_t)cap);
        o.valid = (uint8_t *)realloc(o.valid, (size_t)cap);
        o.orig = (int32_t *)realloc(o.orig, sizeof(int32_t) * (size_t)cap);
      }
      o.ts[o.total] = sub[k];
      o.valid[o.total] = 1;
      o.orig[o.total] = (int32_t)i;
      ++o.total;
    }
  }
  return o;
}

static void free_set(oset *o) {
  free(o->ts); free(o->valid); free(o->orig);
}

int oracle_clip_count(int W, int H, int V, const float *pos, int64_t T, const int32_t *tris, const float *M,
                      int64_t *nsub) {
  int bad = 0;
  ovtx *vs = vertex_stage_all(W, H, V, pos, M);
  oset o = setup_all(W, H, vs, V, T, tris, &bad);
  *nsub = o.total - T;
  free_set(&o);
  free(vs);
  return bad ? ORACLE_BAD_INDEX : ORACLE_OK;
}

/* ------------------------------------------------- O10, brute force over all */
int oracle_raster_brute(int W, int H, int V, const float *pos, int64_t T, const int32_t *tris,
                        const float *M, uint64_t *key, uint32_t *count) {
  int bad = 0;
  ovtx *vs = vertex_stage_all(W, H, V, pos, M);
  oset o = setup_all(W, H, vs, V, T, tris, &bad);
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      uint64_t best = KEY_EMPTY;
      uint32_t n = 0;
      for (int64_t i = 0; i < o.total; ++i) {
        if (!o.valid[i]) continue;
        uint32_t z;
        int64_t w[3];
        if (!cover_and_depth(&o.ts[i], px, py, &z, w)) continue;
        ++n;
        uint64_t k = ((uint64_t)z << 32) | (uint32_t)o.orig[i];
        if (k < best) best = k;
      }
      key[(size_t)py * W + px] = best;
      if (count) count[(size_t)py * W + px] = n;
    }
  free_set(&o); free(vs);
  return bad ? ORACLE_BAD_INDEX : ORACLE_OK;
}

/* Same definition evaluated only at the listed pixels (x, y pairs). */
int oracle_keys_at(int W, int H, int V, const float *pos, int64_t T, const int32_t *tris,
                   const float *M, int64_t npix, const int32_t *pix, uint64_t *key) {
  int bad = 0;
  ovtx *vs = vertex_stage_all(W, H, V, pos, M);
  oset o = setup_all(W, H, vs, V, T, tris, &bad);
  for (int64_t j = 0; j < npix; ++j) {
    int px = pix[2 * j], py = pix[2 * j + 1];
    uint64_t best = KEY_EMPTY;
    for (int64_t i = 0; i < o.total; ++i) {
      if (!o.valid[i]) continue;
      uint32_t z;
      int64_t w[3];
      if (!cover_and_depth(&o.ts[i], px, py, &z, w)) continue;
      uint64_t k = ((uint64_t)z << 32) | (uint32_t)o.orig[i];
      if (k < best) best = k;
    }
    key[j] = best;
  }
  free_set(&o); free(vs);
  return bad ? ORACLE_BAD_INDEX : ORACLE_OK;
}

/* --------------------------------------- bounding-box restricted evaluation
 * Identical output to oracle_raster_brute: a pixel centre outside the
 * bounding box of the snapped vertices lies outside the closed triangle, so
 * some edge function is negative there.  Row bands run on nthreads threads. */
typedef struct {
  int W, H, y0, y1;
  int64_t T;
  const otri *ts;
  const uint8_t *valid;
  const int32_t *orig;
  uint64_t *key;
} band_job;

static int64_t floor_div256(int64_t a) { return a >= 0 ? a / 256 : -((-a + 255) / 256); }

static void *band_worker(void *arg) {
  band_job *j = (band_job *)arg;
  for (int py = j->y0; py < j->y1; ++py)
    for (int px = 0; px < j->W; ++px) j->key[(size_t)py * j->W + px] = KEY_EMPTY;
  for (int64_t i = 0; i < j->T; ++i) {
    if (!j->valid[i]) continue;
    const otri *t = &j->ts[i];
    int64_t xmin = t->X[0], xmax = t->X[0], ymin = t->Y[0], ymax = t->Y[0];
    for (int k = 1; k < 3; ++k) {
      if (t->X[k] < xmin) xmin = t->X[k];
      if (t->X[k] > xmax) xmax = t->X[k];
      if (t->Y[k] < ymin) ymin = t->Y[k];
      if (t->Y[k] > ymax) ymax = t->Y[k];
    }
    /* pixels whose centre 256*p+128 lies in [min, max] */
    int64_t px0 = -floor_div256(-(xmin - 128)), px1 = floor_div256(xmax - 128);
    int64_t py0 = -floor_div256(-(ymin - 128)), py1 = floor_div256(ymax - 128);
    if (px0 < 0) px0 = 0;
    if (px1 > j->W - 1) px1 = j->W - 1;
    if (py0 < j->y0) py0 = j->y0;
    if (py1 > j->y1 - 1) py1 = j->y1 - 1;
    for (int64_t py = py0; py <= py1; ++py)
      for (int64_t px = px0; px <= px1; ++px) {
        uint32_t z;
        int64_t w[3];
        if (!cover_and_depth(t, (int)px, (int)py, &z, w)) continue;
        uint64_t k = ((uint64_t)z << 32) | (uint32_t)j->orig[i];
        uint64_t *dst = &j->key[(size_t)py * j->W + px];
        if (k < *dst) *dst = k;
      }
  }
  return NULL;
}

int oracle_raster_bbox(int W, int H, int V, const float *pos, int64_t T, const int32_t *tris,
                       const float *M, uint64_t *key, int nthreads) {
  int bad = 0;
  ovtx *vs = vertex_stage_all(W, H, V, pos, M);
  oset o = setup_all(W, H, vs, V, T, tris, &bad);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > H) nthreads = H > 0 ? H : 1;
  band_job *jobs = (band_job *)calloc((size_t)nthreads, sizeof(band_job));
  pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int k = 0; k < nthreads; ++k) {
    jobs[k].W = W; jobs[k].H = H; jobs[k].T = o.total; jobs[k].ts = o.ts; jobs[k].valid = o.valid;
    jobs[k].orig = o.orig;
    jobs[k].key = key;
    jobs[k].y0 = (int)((int64_t)H * k / nthreads);
    jobs[k].y1 = (int)((int64_t)H * (k + 1) / nthreads);
  }
  if (nthreads == 1) {
    band_worker(&jobs[0]);
  } else {
    for (int k = 0; k < nthreads; ++k) pthread_create(&th[k], NULL, band_worker, &jobs[k]);
    for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
  }
  free(th); free(jobs); free_set(&o); free(vs);
  return bad ? ORACLE_BAD_INDEX : ORACLE_OK;
}

/* ------------------------------------------------ independent scanline form
 * Per triangle and row, each edge inequality is solved for the interval of
 * pixel columns by exact integer floor/ceil division; depth is evaluated as
 * Z0 + floor((w1*(Z1-Z0) + w2*(Z2-Z0)) / A) with signed 128-bit arithmetic.
 * Written apart from cover_and_depth() so that the two cross-check. */
static int64_t sl_floor_div(int64_t a, int64_t b) { /* b > 0 */
  int64_t q = a / b, r = a % b;
  return (r != 0 && r < 0) ? q - 1 : q;
}
static int64_t sl_ceil_div(int64_t a, int64_t b) { return -sl_floor_div(-a, b); }
static i128 sl_floor_div128(i128 a, i128 b) { /* b > 0 */
  i128 q = a / b, r = a % b;
  return (r != 0 && r < 0) ? q - 1 : q;
}

int oracle_raster_scanline(int W, int H, int V, const float *pos, int64_t T, const int32_t *tris,
                           const float *M, uint64_t *key) {
  int bad = 0;
  ovtx *vs = vertex_stage_all(W, H, V, pos, M);
  oset o = setup_all(W, H, vs, V, T, tris, &bad);
  for (size_t i = 0; i < (size_t)W * H; ++i) key[i] = KEY_EMPTY;
  for (int64_t i = 0; i < o.total; ++i) {
    if (!o.valid[i]) continue;
    const otri t = o.ts[i];
    static const int ea[3] = {1, 2, 0}, eb[3] = {2, 0, 1};
    for (int py = 0; py < H; ++py) {
      int64_t Py = 256 * (int64_t)py + 128;
      int64_t lo = 0, hi = W - 1;
      for (int e = 0; e < 3 && lo <= hi; ++e) {
        int64_t Xa = t.X[ea[e]], Ya = t.Y[ea[e]];
        int64_t dx = t.X[eb[e]] - Xa, dy = t.Y[eb[e]] - Ya;
        int64_t need = (dy < 0 || (dy == 0 && dx > 0)) ? 0 : 1; /* E >= need */
        int64_t c = dx * (Py - Ya) + dy * Xa;                    /* E = c - dy*Px */
        if (dy == 0) {
          if (c < need) hi = lo - 1;
        } else if (dy > 0) { /* Px <= (c - need)/dy */
          int64_t qx = sl_floor_div(c - need, dy);
          int64_t p = sl_floor_div(qx - 128, 256);
          if (p < hi) hi = p;
        } else { /* Px >= (need - c)/(-dy) */
          int64_t qx = sl_ceil_div(need - c, -dy);
          int64_t p = sl_ceil_div(qx - 128, 256);
          if (p > lo) lo = p;
        }
      }
      for (int64_t px = lo; px <= hi; ++px) {
        int64_t Px = 256 * px + 128;
        int64_t w1 = (t.X[0] - t.X[2]) * (Py - t.Y[2]) - (t.Y[0] - t.Y[2]) * (Px - t.X[2]);
        int64_t w2 = (t.X[1] - t.X[0]) * (Py - t.Y[0]) - (t.Y[1] - t.Y[0]) * (Px - t.X[0]);
        i128 num = (i128)w1 * (t.Z[1] - t.Z[0]) + (i128)w2 * (t.Z[2] - t.Z[0]);
        int64_t z = t.Z[0] + (int64_t)sl_floor_div128(num, (i128)t.A);
        uint64_t k = ((uint64_t)z << 32) | (uint32_t)o.orig[i];
        uint64_t *dst = &key[(size_t)py * W + px];
        if (k < *dst) *dst = k;
      }
    }
  }
  free_set(&o);
  free(vs);
  return bad ? ORACLE_BAD_INDEX : ORACLE_OK;
}

/* ---------------------------------------------------------- O12 binary16 */
/* IEEE 754 binary16 from a double, rounding to nearest, ties to even. */
uint16_t oracle_half_from_double(double x) {
  uint16_t sign = signbit(x) ? 0x8000 : 0;
  if (isnan(x)) return (uint16_t)(sign | 0x7E00);
  double a = fabs(x);
  if (a >= 65520.0) return (uint16_t)(sign | 0x7C00); /* halfway to 2^16 and above -> inf */
  if (a == 0.0) return sign;
  int e;
  frexp(a, &e);         /* a = m * 2^e, m in [0.5, 1) */
  int E = e - 1;        /* floor(log2(a)) */
  if (E < -14) E = -14; /* subnormal range shares the quantum 2^-24 */
  double q = ldexp(1.0, E - 10);
  double n = a / q; /* exact: scaling by a power of two */
  double f = floor(n);
  double d = n - f;
  if (d > 0.5 || (d == 0.5 && fmod(f, 2.0) == 1.0)) f += 1.0;
  int64_t r = (int64_t)f;
  if (r < 1024) return (uint16_t)(sign | (uint16_t)r); /* subnormal (E == -14) */
  if (r == 2048) { r = 1024; E += 1; }
  if (E > 15) return (uint16_t)(sign | 0x7C00);
  return (uint16_t)(sign | (uint16_t)((E + 15) << 10) | (uint16_t)(r - 1024));
}

double oracle_double_from_half(uint16_t h) {
  int s = h >> 15, e = (h >> 10) & 31, m = h & 1023;
  double v;
  if (e == 0) v = ldexp((double)m, -24);
  else if (e == 31) v = m ? NAN : INFINITY;
  else v = ldexp((double)(1024 + m), e - 25);
  return s ? -v : v;
}

/* --------------------------------------------------------- O11 shading */
typedef struct {
  double b[3];
  int32_t vid[3];
  uint32_t z;
} winner;

#define FLAG_UNCLAMPED 1
#define FLAG_PERSPECTIVE 2

/* barycentrics of the winning triangle at (px,py), or 0 if key is empty;
 * screen-space (O11), or perspective-correct (O15) when persp is set */
static int pixel_winner_clipped(int W, int H, const ovtx *vs, const int32_t *idx, uint64_t k, int px,
                                int py, winner *o) {
  /* O16: the pixel centre's NDC and the clip-space weights of its ray's
   * point on the triangle's plane */
  double x = ((double)px + 0.5) / (double)W * 2.0 - 1.0;
  double y = 1.0 - ((double)py + 0.5) / (double)H * 2.0;
  double a[3], c[3];
  for (int i = 0; i < 3; ++i) {
    const ovtx *v = &vs[idx[i]];
    a[i] = (double)v->c[0] - x * (double)v->c[3];
    c[i] = (double)v->c[1] - y * (double)v->c[3];
    o->vid[i] = idx[i];
  }
  double n[3] = {a[1] * c[2] - a[2] * c[1], a[2] * c[0] - a[0] * c[2], a[0] * c[1] - a[1] * c[0]};
  double sum = n[0] + n[1] + n[2];
  for (int i = 0; i < 3; ++i) o->b[i] = sum != 0.0 ? n[i] / sum : 1.0 / 3.0;
  o->z = (uint32_t)(k >> 32);
  return 1;
}

static int pixel_winner(int W, int H, const ovtx *vs, int V, const int32_t *tris, uint64_t k, int px, int py,
                        int persp, winner *o) {
  if (k == KEY_EMPTY) return 0;
  uint32_t id = (uint32_t)(k & 0xFFFFFFFFu);
  otri t;
  int bad = 0;
  if (needs_clip(vs, V, tris + 3 * (int64_t)id))
    return pixel_winner_clipped(W, H, vs, tris + 3 * (int64_t)id, k, px, py, o);
  if (!setup_triangle(vs, V, tris + 3 * (int64_t)id, &t, &bad)) return 0;
  int64_t w[3];
  uint32_t z;
  cover_and_depth(&t, px, py, &z, w);
  for (int i = 0; i < 3; ++i) {
    o->b[i] = (double)w[i] / (double)t.A;
    o->vid[i] = t.vid[i];
  }
  if (persp) {
    double q[3], sum = 0.0;
    for (int i = 0; i < 3; ++i) {
      q[i] = o->b[i] / vs[t.vid[i]].w;
      sum += q[i];
    }
    for (int i = 0; i < 3; ++i) o->b[i] = q[i] / sum;
  }
  o->z = (uint32_t)(k >> 32);
  return 1;
}

static const double MATERIAL[3] = {(double)0.80f, (double)0.75f, (double)0.65f};

/* Shading of one pixel.  rgb[3], and for G-buffer output n[3], albedo[3]. */
static void shade_pixel(const winner *wn, const double *color, const double *normal,
                        const double *L, int mode, int unclamped, double rgb[3], double n[3],
                        double alb[3]) {
  for (int c = 0; c < 3; ++c) {
    alb[c] = 0.0;
    n[c] = 0.0;
  }
  for (int i = 0; i < 3; ++i)
    for (int c = 0; c < 3; ++c) {
      if (color) alb[c] += wn->b[i] * color[3 * (size_t)wn->vid[i] + c];
      if (normal) n[c] += wn->b[i] * normal[3 * (size_t)wn->vid[i] + c];
    }
  if (!color)
    for (int c = 0; c < 3; ++c) alb[c] = MATERIAL[c];
  if (mode == 0) {
    for (int c = 0; c < 3; ++c) rgb[c] = alb[c];
  } else if (mode == 1) {
    double d = n[0] * L[0] + n[1] * L[1] + n[2] * L[2];
    double s = unclamped ? d : (d > 0.0 ? d : 0.0);
    for (int c = 0; c < 3; ++c) rgb[c] = alb[c] * s;
  } else {
    for (int c = 0; c < 3; ++c) rgb[c] = 0.0;
  }
}

/* Shades the oracle's own key buffer.  color / normal are [V][3] doubles or
 * NULL; L is [3].  rgba (double [H][W][4]) may be NULL; in mode 2 the
 * G-buffer halves (uint16 [H][W][4]) are written instead. */
int oracle_shade(int W, int H, int V, const float *pos, int64_t T, const int32_t *tris,
                 const float *M, const double *color, const double *normal, const double *L,
                 int mode, int flags, const uint64_t *key, double *rgba, uint16_t *gnormal,
                 uint16_t *galbedo) {
  (void)T;
  const int unclamped = flags & FLAG_UNCLAMPED, persp = (flags & FLAG_PERSPECTIVE) != 0;
  ovtx *vs = vertex_stage_all(W, H, V, pos, M);
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      size_t p = (size_t)py * W + px;
      winner wn;
      double rgb[3] = {0, 0, 0}, n[3] = {0, 0, 0}, alb[3] = {0, 0, 0};
      int hit = pixel_winner(W, H, vs, V, tris, key[p], px, py, persp, &wn);
      if (hit) shade_pixel(&wn, color, normal, L, mode, unclamped, rgb, n, alb);
      if (rgba) {
        for (int c = 0; c < 3; ++c) rgba[4 * p + c] = rgb[c];
        rgba[4 * p + 3] = hit ? 1.0 : 0.0;
      }
      if (gnormal) {
        for (int c = 0; c < 3; ++c) gnormal[4 * p + c] = oracle_half_from_double(hit ? n[c] : 0.0);
        gnormal[4 * p + 3] = 0;
      }
      if (galbedo) {
        for (int c = 0; c < 3; ++c) galbedo[4 * p + c] = oracle_half_from_double(hit ? alb[c] : 0.0);
        galbedo[4 * p + 3] = oracle_half_from_double(hit ? 1.0 : 0.0);
      }
    }
  free(vs);
  return ORACLE_OK;
}

/* ------------------------------------------------------ O12 light pass
 * Per covered pixel, surface point S = (px + 0.5, py + 0.5, z/16777215 * D)
 * with D = max(W, H); for each light l = (x, y, z, I) in index order:
 *   d = P_l - S,  term = I * max(0, n . d/|d|) / (1 + |d|^2 / r^2),
 * r = D/4 (a light at |d| = 0 contributes nothing); rgb = albedo * sum.
 * n and albedo are the binary16 G-buffer values; alpha = 1 when covered. */
int oracle_light_pass(int W, int H, const uint64_t *key, const uint16_t *gnormal,
                      const uint16_t *galbedo, int nlights, const float *lights, double *rgba) {
  double D = (double)(W > H ? W : H);
  double r2 = (0.25 * D) * (0.25 * D);
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      size_t p = (size_t)py * W + px;
      if (key[p] == KEY_EMPTY) {
        for (int c = 0; c < 4; ++c) rgba[4 * p + c] = 0.0;
        continue;
      }
      double z = (double)(uint32_t)(key[p] >> 32);
      double S[3] = {px + 0.5, py + 0.5, z / 16777215.0 * D};
      double n[3], a[3];
      for (int c = 0; c < 3; ++c) {
        n[c] = oracle_double_from_half(gnormal[4 * p + c]);
        a[c] = oracle_double_from_half(galbedo[4 * p + c]);
      }
      double acc = 0.0;
      for (int l = 0; l < nlights; ++l) {
        double d[3] = {lights[4 * l] - S[0], lights[4 * l + 1] - S[1], lights[4 * l + 2] - S[2]};
        double len2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (len2 == 0.0) continue;
        double len = sqrt(len2);
        double ndl = (n[0] * d[0] + n[1] * d[1] + n[2] * d[2]) / len;
        if (ndl < 0.0) ndl = 0.0;
        acc += (double)lights[4 * l + 3] * ndl / (1.0 + len2 / r2);
      }
      for (int c = 0; c < 3; ++c) rgba[4 * p + c] = a[c] * acc;
      rgba[4 * p + 3] = 1.0;
    }
  return ORACLE_OK;
}

/* --------------------------------------------------------- O13 gradients
 * Analytic gradients of a loss with upstream gradient g = dL/drgb (alpha
 * ignored), visibility fixed by the key buffer, accumulated into the
 * outputs.  For Lambert with s = n . L (clamped at 0 unless unclamped):
 *   dL/dc_v += g * s * b_v             (colours, when given)
 *   dL/dn_v += (g . albedo) * b_v * L  (when s > 0 or unclamped)
 *   dL/dL   += (g . albedo) * n
 * and for Gouraud dL/dc_v += g * b_v. */
int oracle_backward(int W, int H, int V, const float *pos, int64_t T, const int32_t *tris,
                    const float *M, const double *color, const double *normal, const double *L,
                    int mode, int flags, const uint64_t *key, const double *dl_drgba,
                    double *dcolor, double *dnormal, double *dlight) {
  (void)T;
  const int unclamped = flags & FLAG_UNCLAMPED, persp = (flags & FLAG_PERSPECTIVE) != 0;
  ovtx *vs = vertex_stage_all(W, H, V, pos, M);
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      size_t p = (size_t)py * W + px;
      winner wn;
      if (!pixel_winner(W, H, vs, V, tris, key[p], px, py, persp, &wn)) continue;
      const double *g = dl_drgba + 4 * p;
      double rgb[3], n[3], alb[3];
      shade_pixel(&wn, color, normal, L, mode, unclamped, rgb, n, alb);
      if (mode == 0) {
        if (dcolor)
          for (int i = 0; i < 3; ++i)
            for (int c = 0; c < 3; ++c) dcolor[3 * (size_t)wn.vid[i] + c] += g[c] * wn.b[i];
        continue;
      }
      if (mode != 1) continue;
      double d = n[0] * L[0] + n[1] * L[1] + n[2] * L[2];
      double s = unclamped ? d : (d > 0.0 ? d : 0.0);
      int active = unclamped || d > 0.0;
      if (dcolor && color)
        for (int i = 0; i < 3; ++i)
          for (int c = 0; c < 3; ++c) dcolor[3 * (size_t)wn.vid[i] + c] += g[c] * s * wn.b[i];
      if (!active) continue;
      double G = g[0] * alb[0] + g[1] * alb[1] + g[2] * alb[2];
      if (dnormal)
        for (int i = 0; i < 3; ++i)
          for (int c = 0; c < 3; ++c) dnormal[3 * (size_t)wn.vid[i] + c] += G * wn.b[i] * L[c];
      if (dlight)
        for (int c = 0; c < 3; ++c) dlight[c] += G * n[c];
    }
  free(vs);
  return ORACLE_OK;
}

/* L = sum over pixels and RGB channels of (rgb - target)^2, float64. */
double oracle_loss(int W, int H, int V, const float *pos, int64_t T, const int32_t *tris,
                   const float *M, const double *color, const double *normal, const double *L,
                   int mode, int flags, const uint64_t *key, const float *target) {
  (void)T;
  const int unclamped = flags & FLAG_UNCLAMPED, persp = (flags & FLAG_PERSPECTIVE) != 0;
  ovtx *vs = vertex_stage_all(W, H, V, pos, M);
  double acc = 0.0;
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      size_t p = (size_t)py * W + px;
      winner wn;
      double rgb[3] = {0, 0, 0}, n[3], alb[3];
      if (pixel_winner(W, H, vs, V, tris, key[p], px, py, persp, &wn))
        shade_pixel(&wn, color, normal, L, mode, unclamped, rgb, n, alb);
      for (int c = 0; c < 3; ++c) {
        double e = rgb[c] - (double)target[4 * p + c];
        acc += e * e;
      }
    }
  free(vs);
  return acc;
}
