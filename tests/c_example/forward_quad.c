/*
 * A plain C caller of the C ABI: rasterizes a full-screen quad (two
 * triangles sharing a diagonal) with Gouraud colours into a 64 x 48
 * framebuffer and checks on the host that every pixel is covered by exactly
 * one of the two triangles (the fill rule leaves no gap or double hit on the
 * shared edge) and that its colour interpolates the vertex colours.
 * Prints "ok" and exits 0 on success.  Build:
 *   gcc -std=c99 forward_quad.c -I<include> -I<cuda>/include \
 *       -L<lib dir> -lpiko_raster -L<cuda>/lib64 -lcudart
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "piko_raster.h"

#define W 64
#define H 48

static int check(int code, piko_raster *h, const char *what) {
  if (code != PIKO_OK) {
    fprintf(stderr, "%s failed: %d (%s)\n", what, code, h ? piko_raster_last_error(h) : "");
    return 1;
  }
  return 0;
}

int main(void) {
  /* NDC corners; red grows with x, green with y, blue constant */
  const float pos[4][4] = {{-1.f, -1.f, 0.f, 1.f}, {1.f, -1.f, 0.f, 1.f}, {1.f, 1.f, 0.f, 1.f}, {-1.f, 1.f, 0.f, 1.f}};
  const float col[4][3] = {{0.f, 0.f, 0.5f}, {1.f, 0.f, 0.5f}, {1.f, 1.f, 0.5f}, {0.f, 1.f, 0.5f}};
  const int32_t tri[2][3] = {{0, 1, 2}, {0, 2, 3}};
  float *d_pos = NULL, *d_col = NULL, *d_rgba = NULL;
  int32_t *d_tri = NULL;
  uint64_t *d_key = NULL;
  if (cudaMalloc((void **)&d_pos, sizeof pos) != cudaSuccess || cudaMalloc((void **)&d_col, sizeof col) != cudaSuccess ||
      cudaMalloc((void **)&d_tri, sizeof tri) != cudaSuccess ||
      cudaMalloc((void **)&d_key, sizeof(uint64_t) * W * H) != cudaSuccess ||
      cudaMalloc((void **)&d_rgba, sizeof(float) * 4 * W * H) != cudaSuccess) {
    fprintf(stderr, "cudaMalloc failed\n");
    return 1;
  }
  cudaMemcpy(d_pos, pos, sizeof pos, cudaMemcpyHostToDevice);
  cudaMemcpy(d_col, col, sizeof col, cudaMemcpyHostToDevice);
  cudaMemcpy(d_tri, tri, sizeof tri, cudaMemcpyHostToDevice);

  piko_raster *h = piko_raster_create(W, H, 16, 16, PIKO_SCHED_HARDWARE);
  if (!h) {
    fprintf(stderr, "piko_raster_create failed\n");
    return 1;
  }
  piko_scene s = {0};
  s.width = W; s.height = H; s.num_vertices = 4; s.num_triangles = 2;
  s.pos = d_pos; s.tris = d_tri; s.color = d_col; s.shade_mode = PIKO_SHADE_GOURAUD;
  piko_framebuffer fb = {0};
  fb.key = d_key; fb.rgba = d_rgba;
  if (check(piko_raster_forward(h, &s, &fb, NULL), h, "forward")) return 1;
  int64_t needed = 0;
  if (check(piko_raster_status(h, &needed), h, "status")) return 1;

  uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * W * H);
  float *rgba = (float *)malloc(sizeof(float) * 4 * W * H);
  cudaMemcpy(key, d_key, sizeof(uint64_t) * W * H, cudaMemcpyDeviceToHost);
  cudaMemcpy(rgba, d_rgba, sizeof(float) * 4 * W * H, cudaMemcpyDeviceToHost);
  int bad = 0;
  for (int y = 0; y < H && !bad; ++y)
    for (int x = 0; x < W; ++x) {
      const size_t p = (size_t)y * W + x;
      const uint32_t id = (uint32_t)(key[p] & 0xFFFFFFFFu);
      /* pixel centre in [0,1]^2, y up as in NDC */
      const float u = (x + 0.5f) / W, v = 1.f - (y + 0.5f) / H;
      if (key[p] == 0xFFFFFFFFFFFFFFFFull || id > 1u || fabsf(rgba[4 * p] - u) > 1e-5f ||
          fabsf(rgba[4 * p + 1] - v) > 1e-5f || fabsf(rgba[4 * p + 2] - 0.5f) > 1e-6f || rgba[4 * p + 3] != 1.f) {
        fprintf(stderr, "pixel (%d, %d): key %llx rgba %g %g %g %g\n", x, y, (unsigned long long)key[p],
                rgba[4 * p], rgba[4 * p + 1], rgba[4 * p + 2], rgba[4 * p + 3]);
        bad = 1;
        break;
      }
    }
  piko_raster_destroy(h);
  cudaFree(d_pos); cudaFree(d_col); cudaFree(d_tri); cudaFree(d_key); cudaFree(d_rgba);
  free(key); free(rgba);
  if (bad) return 1;
  printf("ok\n");
  return 0;
}
