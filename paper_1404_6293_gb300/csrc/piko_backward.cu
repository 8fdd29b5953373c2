// piko_backward.cu -- attribute gradients of one scene through the shading of
// the forward pass: the tile form (a warp per 16 x 16 tile, piko_bwd_tile.cuh)
// and a per-pixel form for scenes of tiny triangles.
#include "piko_bwd_tile.cuh"

namespace piko {

struct BackwardParams {
  BwdScene sc;
  int ntx, ntiles;
};

// Warp form (backward_warp_tile): each warp takes whole tiles, grid-stride.
constexpr int BACKWARD_WARPS = BWD_THREADS / 32;
struct BackwardSmem {
  float stage[BACKWARD_WARPS][BWD_VALS][33];
};
#ifndef PIKO_BWD_MINB
#define PIKO_BWD_MINB 3
#endif
template <bool PERSP, bool CLIP>
__global__ void __launch_bounds__(BWD_THREADS, PIKO_BWD_MINB) k_backward(const __grid_constant__ BackwardParams p) {
  extern __shared__ __align__(16) unsigned char bwd_smem_raw[];
  BackwardSmem& sm = *reinterpret_cast<BackwardSmem*>(bwd_smem_raw);
  const int warp = threadIdx.x >> 5;
  float L0 = 0.f, L1 = 0.f, L2 = 0.f;
  if (p.sc.mode == PIKO_SHADE_LAMBERT) {
    L0 = __ldg(p.sc.light); L1 = __ldg(p.sc.light + 1); L2 = __ldg(p.sc.light + 2);
  }
  const int nwarps = gridDim.x * BACKWARD_WARPS;
  for (int tile = blockIdx.x * BACKWARD_WARPS + warp; tile < p.ntiles; tile += nwarps) {
    const int ty = tile / p.ntx, tx = tile - ty * p.ntx;
    backward_warp_tile<PERSP, CLIP>(p.sc, tx * BWD_TILE_W, ty * BWD_TILE_H, sm.stage[warp], L0, L1, L2);
  }
}
constexpr size_t BACKWARD_SMEM = sizeof(BackwardSmem);

// A winner the vertex stage rejected was clipped (near/far clipping on, pos
// set): its weights are the clip-space ray weights of the pixel centre.
// Per-pixel form, for scenes of tiny triangles (a tile would hold nearly as
// many triangles as pixels, so the tile form's runs are a pixel or two long):
// each warp takes 32 consecutive pixels; lanes whose pixels share a winning
// triangle are summed in shared memory and one lane issues the atomics for
// the group; the light gradient is reduced over the whole CTA.
struct PixelBwdParams {
  int W, H, mode, unclamped;
  int T, V;
  const int* tris;
  const int4* vtx;
  const float* color;
  const float* normal;
  const float* light;
  const float* invw;
  const float4* pos;  // near/far clipping: positions and matrix of clipped winners (NULL: off)
  const float* mvp;
  const unsigned long long* key;
  const float4* dl_drgba;
  float* dcolor;
  float* dnormal;
  float* dlight;
};


constexpr int PIX_THREADS = 256;
constexpr int PIX_VALS = 18;  // per pixel: 3 vertices x (3 colour + 3 normal)

template <bool PERSP>
__global__ void __launch_bounds__(PIX_THREADS) k_backward_pixel(PixelBwdParams p) {
  __shared__ float sval[PIX_THREADS / 32][PIX_VALS][32];
  __shared__ float sred[PIX_THREADS / 32][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  float L0 = 0.f, L1 = 0.f, L2 = 0.f;
  if (p.mode == PIKO_SHADE_LAMBERT) {
    L0 = __ldg(p.light); L1 = __ldg(p.light + 1); L2 = __ldg(p.light + 2);
  }
  float gl0 = 0.f, gl1 = 0.f, gl2 = 0.f;  // this thread's share of dL/dL
  const int npix = p.W * p.H;  // W, H <= 32767
  const int stride = gridDim.x * blockDim.x;
  // warp-uniform trip count so that the warp collectives below stay converged
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < npix; base += stride) {
    const int i = base + lane;
    unsigned long long k = KEY_EMPTY;
    if (i < npix) k = __ldg(p.key + i);
    // a key naming a triangle outside this scene, or one the vertex stage
    // culls, contributes nothing (it cannot come from this scene's forward)
    bool hit = k != KEY_EMPTY && (unsigned)(k & 0xFFFFFFFFu) < (unsigned)p.T;
    unsigned t = hit ? (unsigned)(k & 0xFFFFFFFFu) : 0xFFFFFFFFu;
    TriSetup s;
    bool clipped = false;
    if (hit) {
      const int ia = __ldg(p.tris + 3 * (size_t)t), ib = __ldg(p.tris + 3 * (size_t)t + 1),
                ic = __ldg(p.tris + 3 * (size_t)t + 2);
      const bool in_range = ia >= 0 && ia < p.V && ib >= 0 && ib < p.V && ic >= 0 && ic < p.V;
      hit = in_range && setup_triangle(ia, ib, ic, p.vtx, s);
      if (!hit && in_range && p.pos) {  // a winner the vertex stage rejected was clipped
        clipped = hit = true;
        s.v0 = ia; s.v1 = ib; s.v2 = ic;
      }
      if (!hit) t = 0xFFFFFFFFu;
    }
    float v[PIX_VALS];
#pragma unroll
    for (int q = 0; q < PIX_VALS; ++q) v[q] = 0.f;
    int vid[3] = {0, 0, 0};
    if (hit) {
      const int y = i / p.W, x = i - y * p.W;
      vid[0] = s.v0; vid[1] = s.v1; vid[2] = s.v2;
      float b[3];
      if (clipped) {
        clip_ray_weights(p.pos, p.mvp, p.W, p.H, vid, x, y, b[0], b[1], b[2]);
      } else {
        const long long Px = 256LL * x + 128, Py = 256LL * y + 128;
        const long long w0 = (long long)(s.X2 - s.X1) * (Py - s.Y1) - (long long)(s.Y2 - s.Y1) * (Px - s.X1);
        const long long w1 = (long long)(s.X0 - s.X2) * (Py - s.Y2) - (long long)(s.Y0 - s.Y2) * (Px - s.X2);
        const long long w2 = (long long)(s.X1 - s.X0) * (Py - s.Y0) - (long long)(s.Y1 - s.Y0) * (Px - s.X0);
        const float fA = f32_from_i64(s.A);
        b[0] = __fdiv_rn(f32_from_i64(w0), fA);
        b[1] = __fdiv_rn(f32_from_i64(w1), fA);
        b[2] = __fdiv_rn(f32_from_i64(w2), fA);
        if (PERSP)
          perspective_bary(b[0], b[1], b[2], __ldg(p.invw + vid[0]), __ldg(p.invw + vid[1]), __ldg(p.invw + vid[2]));
      }
      const float4 g = __ldg(p.dl_drgba + i);
      if (p.mode == PIKO_SHADE_GOURAUD) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          v[6 * j + 0] = g.x * b[j]; v[6 * j + 1] = g.y * b[j]; v[6 * j + 2] = g.z * b[j];
        }
      } else {
        float a0 = 0.80f, a1 = 0.75f, a2 = 0.65f;  // material of Listing 1 without colours
        if (p.color) {
          a0 = a1 = a2 = 0.f;
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const float* c = p.color + 3 * (size_t)vid[j];
            a0 += b[j] * __ldg(c); a1 += b[j] * __ldg(c + 1); a2 += b[j] * __ldg(c + 2);
          }
        }
        float n0 = 0.f, n1 = 0.f, n2 = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float* n = p.normal + 3 * (size_t)vid[j];
          n0 += b[j] * __ldg(n); n1 += b[j] * __ldg(n + 1); n2 += b[j] * __ldg(n + 2);
        }
        const float d = n0 * L0 + n1 * L1 + n2 * L2;
        const bool active = p.unclamped || d > 0.f;
        const float sh = p.unclamped ? d : fmaxf(d, 0.f);
        const float G = active ? (g.x * a0 + g.y * a1 + g.z * a2) : 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          if (p.color) {
            v[6 * j + 0] = g.x * sh * b[j]; v[6 * j + 1] = g.y * sh * b[j]; v[6 * j + 2] = g.z * sh * b[j];
          }
          v[6 * j + 3] = G * b[j] * L0; v[6 * j + 4] = G * b[j] * L1; v[6 * j + 5] = G * b[j] * L2;
        }
        gl0 += G * n0; gl1 += G * n1; gl2 += G * n2;
      }
    }
    // group lanes by winning triangle; the lowest lane of each group sums
    // the group's contributions and issues the atomics
    const unsigned grp = __match_any_sync(FULL_MASK, t);
    const bool leader = hit && (grp & lt_mask) == 0u;
    const bool alone = __popc(grp) == 1;
    if (!alone) {
#pragma unroll
      for (int q = 0; q < PIX_VALS; ++q) sval[warp][q][lane] = v[q];
    }
    __syncwarp();
    if (leader) {
      if (!alone) {
        unsigned rest = grp & ~(1u << lane);
        while (rest) {
          const int src = __ffs(rest) - 1;
          rest &= rest - 1;
#pragma unroll
          for (int q = 0; q < PIX_VALS; ++q) v[q] += sval[warp][q][src];
        }
      }
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        if (p.dcolor && (p.mode == PIKO_SHADE_GOURAUD || p.color)) {
          float* dc = p.dcolor + 3 * (size_t)vid[j];
          atomicAdd(dc, v[6 * j]); atomicAdd(dc + 1, v[6 * j + 1]); atomicAdd(dc + 2, v[6 * j + 2]);
        }
        if (p.dnormal && p.mode == PIKO_SHADE_LAMBERT) {
          float* dn = p.dnormal + 3 * (size_t)vid[j];
          atomicAdd(dn, v[6 * j + 3]); atomicAdd(dn + 1, v[6 * j + 4]); atomicAdd(dn + 2, v[6 * j + 5]);
        }
      }
    }
    __syncwarp();
  }
  if (p.dlight && p.mode == PIKO_SHADE_LAMBERT) {
    for (int o = 16; o > 0; o >>= 1) {
      gl0 += __shfl_xor_sync(FULL_MASK, gl0, o);
      gl1 += __shfl_xor_sync(FULL_MASK, gl1, o);
      gl2 += __shfl_xor_sync(FULL_MASK, gl2, o);
    }
    if (lane == 0) { sred[warp][0] = gl0; sred[warp][1] = gl1; sred[warp][2] = gl2; }
    __syncthreads();
    if (threadIdx.x < 3) {
      float acc = 0.f;
      for (int w = 0; w < PIX_THREADS / 32; ++w) acc += sred[w][threadIdx.x];
      atomicAdd(p.dlight + threadIdx.x, acc);
    }
  }
}

using BackwardKernel = void (*)(BackwardParams);

BackwardKernel backward_kernel(bool persp, bool clip) {
  if (persp) return clip ? k_backward<true, true> : k_backward<true, false>;
  return clip ? k_backward<false, true> : k_backward<false, false>;
}

// Blocks of the single-scene backward kernel: as many as fit on the device
// at once, a tile per warp (the shared-memory opt-in is per device, so it is
// cached per device).
int backward_grid(int tiles, int num_sms) {
  static int per_sm_of[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int& per_sm = per_sm_of[dev & 63];
  if (per_sm == 0) {
    int v = 0;
    bool ok = true;
    // the instances share the launch bounds and the shared-memory size
    for (int k = 0; k < 4; ++k)
      ok = ok && cudaFuncSetAttribute(backward_kernel(k & 1, k & 2), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)BACKWARD_SMEM) == cudaSuccess;
    if (!ok ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, backward_kernel(false, false), BWD_THREADS,
                                                      BACKWARD_SMEM) != cudaSuccess ||
        v < 1)
      v = 1;
    per_sm = v;
  }
  long long blocks = (long long)per_sm * num_sms;
  const long long need = (tiles + BACKWARD_WARPS - 1) / BACKWARD_WARPS;
  if (blocks > need) blocks = need;
  return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace piko

using namespace piko;

int piko_backward_launch(int W, int H, int mode, int unclamped, int T, int V, const int* tris, const int4* vtx,
                         const float* color, const float* normal, const float* light, const float* invw,
                         const float* pos, const float* mvp, const unsigned long long* key,
                         const float* dl_drgba, float* dcolor, float* dnormal, float* dlight, int num_sms,
                         cudaStream_t s) {
  const long long npix = (long long)W * H;
#ifndef PIKO_BWD_PIXEL_FORM  // 0: every scene takes the tile form (for comparisons)
#define PIKO_BWD_PIXEL_FORM 1
#endif
  if (PIKO_BWD_PIXEL_FORM && 4LL * T > npix) {
    // more than one triangle per four pixels: triangles of a few pixels
    PixelBwdParams p;
    p.W = W; p.H = H; p.mode = mode; p.unclamped = unclamped; p.T = T; p.V = V;
    p.tris = tris; p.vtx = vtx; p.color = color; p.normal = normal; p.light = light; p.invw = invw;
    p.pos = reinterpret_cast<const float4*>(pos); p.mvp = mvp;
    p.key = key; p.dl_drgba = reinterpret_cast<const float4*>(dl_drgba);
    p.dcolor = dcolor; p.dnormal = dnormal; p.dlight = dlight;
    long long blocks = (npix + PIX_THREADS - 1) / PIX_THREADS;
    if (blocks > (long long)num_sms * 4) blocks = (long long)num_sms * 4;
    if (blocks < 1) blocks = 1;
    if (invw)
      k_backward_pixel<true><<<(int)blocks, PIX_THREADS, 0, s>>>(p);
    else
      k_backward_pixel<false><<<(int)blocks, PIX_THREADS, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
  }
  BackwardParams p;
  BwdScene& c = p.sc;
  c.W = W; c.H = H; c.mode = mode; c.unclamped = unclamped; c.T = T; c.V = V;
  c.tris = tris; c.vtx = vtx; c.color = color; c.normal = normal; c.light = light; c.invw = invw;
  c.pos = reinterpret_cast<const float4*>(pos); c.mvp = mvp;
  c.key = key; c.dl = reinterpret_cast<const float4*>(dl_drgba);
  c.dcolor = dcolor; c.dnormal = dnormal; c.dlight = dlight;
  p.ntx = (W + BWD_TILE_W - 1) / BWD_TILE_W;
  p.ntiles = p.ntx * ((H + BWD_TILE_H - 1) / BWD_TILE_H);
  const int blocks = backward_grid(p.ntiles, num_sms);
  backward_kernel(invw != nullptr, pos != nullptr)<<<blocks, BWD_THREADS, BACKWARD_SMEM, s>>>(p);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
