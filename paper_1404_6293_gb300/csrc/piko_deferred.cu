// piko_deferred.cu -- per-pixel light pass over a G-buffer (deferred shading).
//
// Shader complexity measured in number of lights is the axis of the
// paper's Fig. (a) in Sec. 7.2; the supplementary deferred-shading raster
// pipeline the paper mentions in Sec. 7.1 is not printed, so the light model
// is this library's:
//   S = (x + 0.5, y + 0.5, depth / (2^24 - 1) * D),  D = max(W, H),  r = D / 4
//   rgb = albedo * sum_l I_l * max(0, n . (P_l - S) / |P_l - S|) / (1 + |P_l - S|^2 / r^2)
// with n and albedo read from the binary16 G-buffer.  The pass is FP32-ALU
// bound (about 20 operations per pixel and light); lights live in shared
// memory and every thread shades whole pixels.
#include <cuda_fp16.h>

#include "piko_internal.cuh"

namespace piko {

__device__ __forceinline__ float4 unpack_half4(uint2 v) {
  const __half2 lo = *reinterpret_cast<const __half2*>(&v.x);
  const __half2 hi = *reinterpret_cast<const __half2*>(&v.y);
  const float2 a = __half22float2(lo), b = __half22float2(hi);
  return make_float4(a.x, a.y, b.x, b.y);
}

__global__ void __launch_bounds__(256) k_deferred_light(int W, int H, const unsigned long long* __restrict__ key,
                                                        const uint2* __restrict__ gnorm,
                                                        const uint2* __restrict__ galb,
                                                        const float4* __restrict__ lights, int n_lights,
                                                        float4* __restrict__ rgba) {
  extern __shared__ float4 slights[];
  for (int i = threadIdx.x; i < n_lights; i += blockDim.x) slights[i] = lights[i];
  __syncthreads();
  const float D = (float)max(W, H);
  const float inv_r2 = 1.0f / ((0.25f * D) * (0.25f * D));
  const float zscale = D / 16777215.0f;
  const int npix = W * H;  // W, H <= 32767
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
    const unsigned long long k = __ldg(key + i);
    if (k == KEY_EMPTY) {
      rgba[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    const int y = i / W, x = i - y * W;
    const float4 n = unpack_half4(__ldg(gnorm + i));
    const float4 a = unpack_half4(__ldg(galb + i));
    const float sx = (float)x + 0.5f, sy = (float)y + 0.5f;
    const float sz = (float)(unsigned)(k >> 32) * zscale;
    float acc0 = 0.f, acc1 = 0.f;
    int l = 0;
    for (; l + 1 < n_lights; l += 2) {
      const float4 p = slights[l], q = slights[l + 1];
      const float dx = p.x - sx, dy = p.y - sy, dz = p.z - sz;
      const float ex = q.x - sx, ey = q.y - sy, ez = q.z - sz;
      const float d2 = dx * dx + dy * dy + dz * dz, e2 = ex * ex + ey * ey + ez * ez;
      const float nd = n.x * dx + n.y * dy + n.z * dz, ne = n.x * ex + n.y * ey + n.z * ez;
      // fast reciprocal square root and division (2 ulp each): a light's
      // term is O(1/16), so 64 of them stay far inside the 1e-5 tolerance
      if (d2 > 0.f && nd > 0.f) acc0 += __fdividef(p.w * nd * rsqrtf(d2), 1.0f + d2 * inv_r2);
      if (e2 > 0.f && ne > 0.f) acc1 += __fdividef(q.w * ne * rsqrtf(e2), 1.0f + e2 * inv_r2);
    }
    if (l < n_lights) {
      const float4 p = slights[l];
      const float dx = p.x - sx, dy = p.y - sy, dz = p.z - sz;
      const float d2 = dx * dx + dy * dy + dz * dz;
      const float nd = n.x * dx + n.y * dy + n.z * dz;
      if (d2 > 0.f && nd > 0.f) acc0 += __fdividef(p.w * nd * rsqrtf(d2), 1.0f + d2 * inv_r2);
    }
    const float acc = acc0 + acc1;
    rgba[i] = make_float4(a.x * acc, a.y * acc, a.z * acc, 1.0f);
  }
}

void launch_deferred_light(int W, int H, const unsigned long long* key, const uint2* gnorm, const uint2* galb,
                           const float4* lights, int n_lights, float4* rgba, int num_sms, cudaStream_t s) {
  const long long npix = (long long)W * H;
  long long blocks = (npix + 255) / 256;
  if (blocks > (long long)num_sms * 8) blocks = (long long)num_sms * 8;
  if (blocks < 1) blocks = 1;
  k_deferred_light<<<(int)blocks, 256, (size_t)n_lights * sizeof(float4), s>>>(W, H, key, gnorm, galb, lights,
                                                                               n_lights, rgba);
}

}  // namespace piko
