// piko_scan.cuh -- exclusive scan of the per-bin counts into CSR offsets,
// one chunk of blockDim.x * SCAN_PER bins per call, shared by the
// single-scene scan kernel and the batch kernel.
//
// A single-pass decoupled look-back scan: chunks are taken in ticket order,
// so every predecessor of a chunk has started.  Each chunk publishes its
// aggregate, then its inclusive prefix, in a 64-bit state word tagged with
// the frame's epoch (so the words never need clearing):
//   bits 63..62 kind (1 aggregate, 2 inclusive prefix), 61..46 epoch, 45..0 value.
// off[b] = entries of all earlier bins; the scatter cursor of a bin starts
// after its single-bin part; both count arrays are zeroed for the next frame.
// A look-back wait is bounded by a clock budget (wait_budget cycles, by
// default WAIT_BUDGET_CYCLES); on expiry the scan records PIKO_ERR_TIMEOUT
// and the frame's later stages skip their work.  TEST_WITHHOLD_SCAN in
// `withhold` makes chunk 0 keep its state unpublished, so that the next
// chunk's wait runs out: a test of that path, which faults nothing.
#pragma once

#include "piko_internal.cuh"

namespace piko {

constexpr int SCAN_PER = 8;
// CTA size of the single-scene scan (k_scan): one CTA per chunk of
// FWD_SCAN_CHUNK bins.  (1024 threads, which make a 1080p frame at 16 x 16
// one chunk with no look-back, measured slower: 11.1 against 8.0 us.)
#ifndef PIKO_SCAN_THREADS
#define PIKO_SCAN_THREADS 256
#endif
constexpr int FWD_SCAN_THREADS = PIKO_SCAN_THREADS;
constexpr int FWD_SCAN_CHUNK = FWD_SCAN_THREADS * SCAN_PER;
constexpr unsigned long long SCAN_KIND_AGG = 1ull << 62, SCAN_KIND_PREFIX = 2ull << 62;
constexpr unsigned long long SCAN_VALUE_MASK = (1ull << 46) - 1ull;
constexpr long long WAIT_BUDGET_CYCLES = 40000000;  // ~20 ms at 2 GHz
// test hooks (bits of the `withhold` argument)
constexpr int TEST_WITHHOLD_SCAN = 1;     // scan chunk 0 does not publish its state
constexpr int TEST_WITHHOLD_BARRIER = 2;  // batch CTA 0 does not arrive at the first grid barrier
constexpr int TEST_WITHHOLD_HEAVY = 4;    // the heavy-triangle list of AssignBin counts as full

struct ScanSmem {
  unsigned long long warp_sums[32];
  unsigned long long excl;
  int chunk;
};

__device__ __forceinline__ void load8(const unsigned* __restrict__ a, int b0, int nbins, bool vec, unsigned* v) {
  if (vec && b0 + 8 <= nbins) {
    const uint4 x = __ldcg(reinterpret_cast<const uint4*>(a + b0)), y = __ldcg(reinterpret_cast<const uint4*>(a + b0 + 4));
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w; v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = b0 + j < nbins ? __ldcg(a + b0 + j) : 0u;
  }
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Scans chunk `chunk` of nchunks (all threads of the CTA call it; it
// contains barriers).  The last chunk writes the total, checks the capacity
// and resets *queue_to_reset (the Process stage's tile queue).
__device__ __forceinline__ void scan_chunk(int chunk, int nchunks, int nbins, unsigned* __restrict__ cnt,
                                           unsigned* __restrict__ bin_off, unsigned* __restrict__ cursor,
                                           unsigned long long capacity, DevStatus* st,
                                           unsigned long long* __restrict__ chunk_state, unsigned epoch, ScanSmem& sm,
                                           unsigned* queue_to_reset, long long wait_budget = WAIT_BUDGET_CYCLES,
                                           int withhold = 0) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  const unsigned long long tag = (unsigned long long)(epoch & 0xFFFFu) << 46;
  unsigned* __restrict__ multi = cnt + nbins;
  const bool vec = (nbins & 3) == 0;  // second array 16-byte aligned
  const int b0 = chunk * (int)blockDim.x * SCAN_PER + tid * SCAN_PER;
  unsigned sg[SCAN_PER], mu[SCAN_PER];
  load8(cnt, b0, nbins, vec, sg);
  load8(multi, b0, nbins, vec, mu);
  unsigned long long local = 0;
#pragma unroll
  for (int j = 0; j < SCAN_PER; ++j) local += (unsigned long long)sg[j] + mu[j];
  unsigned long long v = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(FULL_MASK, v, o);
    if (lane >= o) v += u;
  }
  if (lane == 31) sm.warp_sums[w] = v;
  __syncthreads();
  if (w == 0) {
    unsigned long long x = lane < nw ? sm.warp_sums[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long u = __shfl_up_sync(FULL_MASK, x, o);
      if (lane >= o) x += u;
    }
    if (lane < nw) sm.warp_sums[lane] = x;
  }
  __syncthreads();
  const unsigned long long agg = sm.warp_sums[nw - 1];
  if (tid == 0) {
    unsigned long long excl = 0;
    if (chunk == 0) {
      if (!(withhold & TEST_WITHHOLD_SCAN)) st_release_u64(chunk_state, SCAN_KIND_PREFIX | tag | (agg & SCAN_VALUE_MASK));
    } else {
      st_release_u64(chunk_state + chunk, SCAN_KIND_AGG | tag | (agg & SCAN_VALUE_MASK));
      const long long t0 = clock64();
      bool timed_out = false;
      for (int j = chunk - 1; j >= 0 && !timed_out;) {
        const unsigned long long sv = ld_acquire_u64(chunk_state + j);
        const unsigned long long sv_epoch = sv & ~SCAN_VALUE_MASK & ~(3ull << 62);
        if (sv_epoch != tag || (sv >> 62) == 0) {
          if (clock64() - t0 > wait_budget) timed_out = true;
          else __nanosleep(64);
          continue;  // predecessor not published for this frame yet
        }
        excl += sv & SCAN_VALUE_MASK;
        if ((sv >> 62) == 2) break;  // inclusive prefix: done
        --j;
      }
      if (timed_out) record_error(st, PIKO_ERR_TIMEOUT);
      st_release_u64(chunk_state + chunk, SCAN_KIND_PREFIX | tag | ((excl + agg) & SCAN_VALUE_MASK));
    }
    sm.excl = excl;
  }
  __syncthreads();
  unsigned long long run = sm.excl + v - local + (w > 0 ? sm.warp_sums[w - 1] : 0ull);
  unsigned of[SCAN_PER], cu[SCAN_PER];
#pragma unroll
  for (int j = 0; j < SCAN_PER; ++j) {
    of[j] = (unsigned)run;
    cu[j] = (unsigned)(run + sg[j]);
    run += (unsigned long long)sg[j] + mu[j];
  }
  if (vec && b0 + SCAN_PER <= nbins) {
    reinterpret_cast<uint4*>(bin_off + b0)[0] = make_uint4(of[0], of[1], of[2], of[3]);
    reinterpret_cast<uint4*>(bin_off + b0)[1] = make_uint4(of[4], of[5], of[6], of[7]);
    reinterpret_cast<uint4*>(cursor + b0)[0] = make_uint4(cu[0], cu[1], cu[2], cu[3]);
    reinterpret_cast<uint4*>(cursor + b0)[1] = make_uint4(cu[4], cu[5], cu[6], cu[7]);
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    reinterpret_cast<uint4*>(cnt + b0)[0] = z;
    reinterpret_cast<uint4*>(cnt + b0)[1] = z;
    reinterpret_cast<uint4*>(multi + b0)[0] = z;
    reinterpret_cast<uint4*>(multi + b0)[1] = z;
  } else {
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j)
      if (b0 + j < nbins) {
        bin_off[b0 + j] = of[j];
        cursor[b0 + j] = cu[j];
        cnt[b0 + j] = 0u;
        multi[b0 + j] = 0u;
      }
  }
  if (chunk == nchunks - 1 && tid == 0) {
    const unsigned long long total = sm.excl + agg;
    const bool ok = total <= capacity;
    if (ok) bin_off[nbins] = (unsigned)total;
    st->needed = total;
    *queue_to_reset = 0u;
    if (!ok) record_error(st, PIKO_ERR_OVERFLOW);
  }
}

}  // namespace piko
