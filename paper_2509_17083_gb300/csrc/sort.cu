// Tile binning and depth ordering (Sec. 3.1: Gaussians are ordered by depth
// and composited per pixel). Instances carry the 64-bit key
// (tile << 32) | float_bits(depth); their stable order is produced by LSD
// radix passes: four 8-bit passes over the 32 depth bits of the visible
// Gaussians (here, or beforehand by hyrf_depth_order from the positions),
// emission of each Gaussian's tiles in that order, then the tile bits over
// the instances (split evenly over the passes). Every pass is
// reduce-then-scan (histogram, per-digit column scan, stable scatter), so
// no kernel waits on another CTA.
#include "footprint.cuh"

namespace hyrf {

constexpr int kRT = 256;         // radix threads per CTA
constexpr int kSub = 2048;       // elements per scatter sub-tile (8 warps x 8 rounds x 32)
constexpr int kRounds = kSub / 256;
constexpr int kMaxRadixCTAs = 2048;
// Elements per radix CTA (the CTA count is the capacity over this, at most
// kMaxRadixCTAs) and the scatter's resident CTAs per SM (its register cap).
#ifndef HYRF_RADIX_PER_CTA
#define HYRF_RADIX_PER_CTA 2048
#endif
#ifndef HYRF_RADIX_SCATTER_CTAS
#define HYRF_RADIX_SCATTER_CTAS 5
#endif

__device__ __forceinline__ int dev_chunk(int n, int G) {
  int c = (n + G - 1) / G;
  return (c + kSub - 1) / kSub * kSub;
}

__device__ __forceinline__ int clamp_n(const int32_t* n_ptr, int cap) {
  int n = *n_ptr;
  return n < 0 ? 0 : (n > cap ? cap : n);
}

__global__ void __launch_bounds__(kRT) k_radix_hist(const uint32_t* __restrict__ keys,
                                                    const int32_t* __restrict__ n_ptr, int cap,
                                                    int shift, uint32_t mask,
                                                    uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  const int G = gridDim.x, b = blockIdx.x;
  h[threadIdx.x] = 0;
  __syncthreads();
  const int n = clamp_n(n_ptr, cap);
  const int chunk = dev_chunk(n, G);
  const int64_t start = (int64_t)b * chunk;
  const int64_t end = (start + chunk < (int64_t)n) ? start + chunk : (int64_t)n;
  for (int64_t i = start + threadIdx.x; i < end; i += kRT) atomicAdd(&h[(keys[i] >> shift) & mask], 1u);
  __syncthreads();
  if (threadIdx.x <= mask) hist[threadIdx.x * G + b] = h[threadIdx.x];  // the pass's digits only
}

// One CTA per digit of the pass (mask + 1 of them): exclusive scan of the
// digit's column over the G CTAs; digit totals to totals[d]. Entries of
// hist and totals past the pass's digits are left as they are: the
// scatter's digit bases below mask + 1 do not depend on them.
__global__ void __launch_bounds__(kRT) k_radix_colscan(uint32_t* __restrict__ hist, int G,
                                                       uint32_t* __restrict__ totals) {
  __shared__ uint32_t wsum[kRT / 32];
  uint32_t* col = hist + (size_t)blockIdx.x * G;
  const int per = (G + kRT - 1) / kRT;
  const int s0 = threadIdx.x * per;
  uint32_t v[kMaxRadixCTAs / kRT];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < kMaxRadixCTAs / kRT; ++k) {
    v[k] = (k < per && s0 + k < G) ? col[s0 + k] : 0u;
    sum += v[k];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = sum;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  uint32_t before = 0, total = 0;
  for (int j = 0; j < kRT / 32; ++j) {
    before += j < w ? wsum[j] : 0u;
    total += wsum[j];
  }
  uint32_t run = before + x - sum;
#pragma unroll
  for (int k = 0; k < kMaxRadixCTAs / kRT; ++k) {
    if (k < per && s0 + k < G) col[s0 + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kRT, HYRF_RADIX_SCATTER_CTAS) k_radix_scatter(const uint32_t* __restrict__ keys_in,
                                                       const int32_t* __restrict__ vals_in,
                                                       uint32_t* __restrict__ keys_out,
                                                       int32_t* __restrict__ vals_out,
                                                       const int32_t* __restrict__ n_ptr, int cap,
                                                       int shift, uint32_t mask,
                                                       const uint32_t* __restrict__ hist,
                                                       const uint32_t* __restrict__ totals) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t sub_total[256];
  __shared__ uint32_t lstart[256];   // digit starts within the sub-tile
  __shared__ uint32_t whist[8][256];
  __shared__ uint32_t wsum[8];
  __shared__ uint32_t sk[kSub];      // the sub-tile in digit order
  __shared__ int32_t sv[kSub];
  const int G = gridDim.x, b = blockIdx.x, t = threadIdx.x;
  const int lane = t & 31, w = t >> 5;
  // digit base = exclusive scan of the digit totals + this CTA's column prefix
  {
    const uint32_t tot = t <= (int)mask ? totals[t] : 0u;  // (only the pass's digits were written)
    uint32_t x = tot;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int j = 0; j < w; ++j) before += wsum[j];
    base[t] = before + x - tot + (t <= (int)mask ? hist[t * G + b] : 0u);
#pragma unroll
    for (int j = 0; j < 8; ++j) whist[j][t] = 0;
  }
  __syncthreads();
  const int n = clamp_n(n_ptr, cap);
  const int chunk = dev_chunk(n, G);
  const int64_t start = (int64_t)b * chunk;
  const int64_t end = (start + chunk < (int64_t)n) ? start + chunk : (int64_t)n;
  for (int64_t sub = start; sub < end; sub += kSub) {
    // (a round's validity and digits are recomputed where needed: fewer
    // registers, more CTAs per SM)
    uint32_t key[kRounds], rank[kRounds];
    int32_t val[kRounds];
    const int64_t idx0 = sub + w * (32 * kRounds) + lane;  // round r: idx0 + 32 r
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      const int64_t idx = idx0 + r * 32;
      const bool valid = idx < end;
      key[r] = valid ? keys_in[idx] : 0u;
      val[r] = valid ? vals_in[idx] : 0;
      const uint32_t dig = (key[r] >> shift) & mask;
      const uint32_t m_valid = __ballot_sync(0xffffffffu, valid);
      const uint32_t peers = __match_any_sync(0xffffffffu, valid ? dig : 0x10000u + lane) & m_valid;
      uint32_t prev = 0;
      if (valid) prev = whist[w][dig];
      __syncwarp();
      rank[r] = prev + __popc(peers & ((1u << lane) - 1u));
      if (valid && lane == __ffs(peers) - 1) whist[w][dig] = prev + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    uint32_t tot;
    {
      uint32_t run = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t c = whist[j][t];
        whist[j][t] = run;
        run += c;
      }
      sub_total[t] = run;
      tot = run;
    }
    // exclusive scan of the digit counts: where each digit starts in the
    // sub-tile
    {
      uint32_t x = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) wsum[w] = x;
      __syncthreads();
      uint32_t before = 0;
      for (int j = 0; j < w; ++j) before += wsum[j];
      lstart[t] = before + x - tot;
    }
    __syncthreads();
    // stage the sub-tile in digit order, then write each digit's run to
    // consecutive global positions (coalesced)
#pragma unroll
    for (int r = 0; r < kRounds; ++r) {
      if (idx0 + r * 32 >= end) continue;
      const uint32_t dig = (key[r] >> shift) & mask;
      const uint32_t lp = lstart[dig] + whist[w][dig] + rank[r];
      sk[lp] = key[r];
      sv[lp] = val[r];
    }
    __syncthreads();
    const int cnt = (int)((end - sub) < kSub ? (end - sub) : kSub);
    for (int i = t; i < cnt; i += kRT) {
      const uint32_t k = sk[i];
      const uint32_t d = (k >> shift) & mask;
      const uint32_t pos = base[d] + ((uint32_t)i - lstart[d]);
      keys_out[pos] = k;
      vals_out[pos] = sv[i];
    }
    __syncthreads();
    base[t] += sub_total[t];
#pragma unroll
    for (int j = 0; j < 8; ++j) whist[j][t] = 0;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- scan of tile counts

constexpr int kScanChunk = 2048;  // elements per scan CTA (256 threads x 8)

__device__ __forceinline__ int tiles_of_sorted(const int32_t* ntiles, const int32_t* order, int j,
                                               int n) {
  const int g = order[j];
  return (g >= 0 && g < n) ? ntiles[g] : 0;
}

__global__ void __launch_bounds__(256) k_count_sums(const int32_t* __restrict__ ntiles,
                                                    const int32_t* __restrict__ order,
                                                    const int32_t* __restrict__ n_ptr, int cap,
                                                    int64_t* __restrict__ sums) {
  const int n = clamp_n(n_ptr, cap);
  const int64_t start = (int64_t)blockIdx.x * kScanChunk;
  int64_t s = 0;
  for (int k = 0; k < kScanChunk / 256; ++k) {
    const int64_t j = start + k * 256 + threadIdx.x;
    if (j < n) s += tiles_of_sorted(ntiles, order, (int)j, cap);
  }
  __shared__ int64_t red[8];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < 8; ++w) t += red[w];
    sums[blockIdx.x] = t;
  }
}

// Exclusive scan of the CTA sums; writes K = min(total, capacity) and the
// overflow flag.
__global__ void __launch_bounds__(1024) k_scan_sums(int64_t* __restrict__ sums, int m,
                                                    int64_t capacity, int32_t* __restrict__ n_inst,
                                                    int32_t* status) {
  __shared__ int64_t wsums[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < m; base += 1024) {
    const int i = base + threadIdx.x;
    const int64_t v = i < m ? sums[i] : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsums[w] = x;
    __syncthreads();
    if (w == 0) {
      int64_t s = wsums[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      wsums[lane] = s;
    }
    __syncthreads();
    const int64_t incl = x + (w > 0 ? wsums[w - 1] : 0) + carry;
    if (i < m) sums[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (carry > capacity) set_status(status, HYRF_ERR_OVERFLOW);
    *n_inst = (int32_t)(carry < capacity ? carry : capacity);
  }
}

// Instance offset of every sorted Gaussian: the chunk's base (k_scan_sums)
// plus the exclusive scan of the tile counts inside the chunk. off[n] = K
// (unclamped total, saturated to 32 bits).
__global__ void __launch_bounds__(256) k_offsets(const int32_t* __restrict__ ntiles,
                                                 const int32_t* __restrict__ order,
                                                 const int32_t* __restrict__ n_ptr, int cap_n,
                                                 const int64_t* __restrict__ sums, int nchunks,
                                                 uint32_t* __restrict__ off) {
  __shared__ int64_t wsum[8];
  const int n = clamp_n(n_ptr, cap_n);
  const int64_t start = (int64_t)blockIdx.x * kScanChunk;
  int64_t run = sums[blockIdx.x];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int k = 0; k < kScanChunk / 256; ++k) {
    const int64_t j = start + k * 256 + t;
    const int c = j < n ? tiles_of_sorted(ntiles, order, (int)j, cap_n) : 0;
    int64_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int64_t before = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      before += q < w ? wsum[q] : 0;
      tot += wsum[q];
    }
    const int64_t o = run + before + x - c;
    if (j < n) off[j] = (uint32_t)(o < 0xffffffffll ? o : 0xffffffffll);
    run += tot;
    __syncthreads();
  }
  if (blockIdx.x == nchunks - 1 && t == 0) off[n] = (uint32_t)(run < 0xffffffffll ? run : 0xffffffffll);
}

// Largest index i in [lo, hi] with a[i] <= e (a non-decreasing, a[lo] <= e).
template <class A>
__device__ __forceinline__ int last_le(const A& a, int lo, int hi, uint32_t e) {
  ++hi;  // a[hi] > e or hi one past the range
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

// last_le of two values at once by the whole CTA: threads [0, 128) search
// v[0], threads [128, 256) v[1], each round probing 128 evenly spaced
// positions of the current interval (three rounds for two million entries,
// instead of twenty dependent loads). Result in res[0], res[1].
__device__ __forceinline__ void last_le2_cta(const uint32_t* __restrict__ a, int n, uint32_t v0, uint32_t v1,
                                             int* res) {
  __shared__ int lo[2], hi[2], best[2];
  const int t = threadIdx.x, q = t >> 7, i = t & 127;
  if (t < 2) {
    lo[t] = 0;
    hi[t] = n - 1;
  }
  __syncthreads();
  for (;;) {
    const int l = lo[q], h = hi[q];
    const bool more = h > l;
    if (i == 0) best[q] = 0;
    __syncthreads();
    if (more) {
      const int64_t span = (int64_t)h - l + 1;
      const int pos = l + (int)(span * i / 128);
      if (a[pos] <= (q ? v1 : v0)) atomicMax(&best[q], i);
    }
    __syncthreads();
    if (i == 0 && more) {
      const int64_t span = (int64_t)h - l + 1;
      const int b = best[q];
      lo[q] = l + (int)(span * b / 128);
      hi[q] = b < 127 ? l + (int)(span * (b + 1) / 128) - 1 : h;
      if (hi[q] < lo[q]) hi[q] = lo[q];
    }
    __syncthreads();
    if (lo[0] == hi[0] && lo[1] == hi[1]) break;  // CTA-uniform
  }
  if (t < 2) res[t] = lo[t];
}

constexpr int kExpandItems = 2048;  // instances per CTA
constexpr int kExpandSlice = 2048;  // sorted Gaussians cached per CTA
constexpr int kExpandRows = 2048;   // footprint tile rows cached per CTA
constexpr int kExpandPer = kExpandItems / 256;  // instances per thread (packed footprints)

// Offset from x0 and length of row j's span in a packed footprint record
// (words 1..8 of the record: wa, wb; footprint.cuh).
__device__ __forceinline__ void span_at(const uint4& wa, const uint4& wb, int j, int& off, int& len) {
  const int k = j >> 1;
  uint32_t w = wa.x;
  w = k == 1 ? wa.y : w;
  w = k == 2 ? wa.z : w;
  w = k == 3 ? wa.w : w;
  w = k == 4 ? wb.x : w;
  w = k == 5 ? wb.y : w;
  w = k == 6 ? wb.z : w;
  w = k == 7 ? wb.w : w;
  const uint32_t h = (w >> (16 * (j & 1))) & 0xffffu;
  off = (int)(h & 0xffu);
  len = (int)(h >> 8);
}

// Exclusive prefix sums of a[0, n) in place, n <= 2048, by a 256-thread CTA
// (eight consecutive entries per thread); a[n] = the total, also returned.
// Called by every thread of the CTA.
__device__ __forceinline__ uint32_t cta_excl_scan2048(uint32_t* a, int n, uint32_t* wsum) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  uint32_t v[8], s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = 8 * t + q;
    v[q] = i < n ? a[i] : 0u;
    s += v[q];
  }
  uint32_t inc = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  uint32_t run = inc - s, tot = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const uint32_t x = wsum[q];
    if (q < w) run += x;
    tot += x;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int i = 8 * t + q;
    if (i < n) a[i] = run;
    run += v[q];
  }
  if (t == 0) a[n] = tot;
  __syncthreads();
  return tot;
}

// Each CTA writes a fixed range of instances (balanced however unequal the
// Gaussians' footprints are): it finds the sorted Gaussians that own its
// range, caches their offsets, and its threads write consecutive instances
// (coalesced), each finding its owner by binary search. Instance r of a
// Gaussian with rectangle [x0, x1) x [y0, y1) is tile (y0 + r / w, x0 + r % w):
// row-major order.
__global__ void __launch_bounds__(256) k_expand(const int32_t* __restrict__ rect,
                                                const int32_t* __restrict__ order,
                                                const int32_t* __restrict__ n_ptr, int cap_n,
                                                const uint32_t* __restrict__ off,
                                                const int32_t* __restrict__ k_ptr, int cap_k, int TX,
                                                uint32_t* __restrict__ tile_keys,
                                                int32_t* __restrict__ tile_vals,
                                                const float2* __restrict__ mean2d,
                                                const float4* __restrict__ foot) {
  __shared__ uint32_t soff[kExpandSlice + 1];
  __shared__ int32_t sid[kExpandSlice];
  __shared__ int range[2];
  const int n = clamp_n(n_ptr, cap_n);
  const int K = clamp_n(k_ptr, cap_k);
  const int64_t e0 = (int64_t)blockIdx.x * kExpandItems;
  if (e0 >= K || n == 0) return;  // CTA-uniform
  const int e1 = (int)(e0 + kExpandItems < K ? e0 + kExpandItems : K);
  const int t = threadIdx.x;
  last_le2_cta(off, n, (uint32_t)e0, (uint32_t)(e1 - 1), range);
  __syncthreads();
  const int jlo = range[0], jhi = range[1];
  const int L = jhi - jlo + 1;
  const bool cached = L <= kExpandSlice;
  if (cached) {
    for (int i = t; i < L; i += 256) {
      soff[i] = off[jlo + i];
      sid[i] = order[jlo + i];
    }
    if (t == 0) soff[L] = off[jhi + 1];
  }
  __syncthreads();
  if (foot) {
    // footprints. Packed records: each instance's tile from the row spans
    // the projection stored. Otherwise one thread per (Gaussian, tile row)
    // of the CTA's range computes the row's span (footprint.cuh: the spans
    // the projection counted), a scan of the span lengths gives each row's
    // first instance, and each row writes its instances.
    __shared__ uint32_t rstart[kExpandRows + 1];
    __shared__ uint32_t rtile[kExpandRows];
    __shared__ int32_t rg[kExpandRows];
    __shared__ uint32_t wsum[8];
    if (cached) {
      // eight consecutive instances per thread: one search of the cached
      // offsets finds the first one's Gaussian and a walk of its packed row
      // spans (footprint.cuh) its row; the thread then steps along the
      // spans, and to the next Gaussian, instance by instance. Keys and
      // values are staged in shared memory and written out coalesced. A
      // CTA whose range holds an unpacked record redoes the range below.
      static_assert(kExpandRows >= kExpandItems, "staging");
      bool unpacked = false;
      const int q0 = (int)e0 + kExpandPer * t, q1 = min(q0 + kExpandPer, e1);
      if (q0 < q1) {
        int i = last_le(soff, 0, L - 1, (uint32_t)q0);
        int rg_ = q0 - (int)soff[i];  // instance index within Gaussian i
        int g = 0, cnt = 0, x0 = 0, y0 = 0, rows = 0, j = 0, c = 0, off = 0, len = 0;
        bool ok = false;
        uint4 wa = make_uint4(0u, 0u, 0u, 0u), wb = wa;
        auto load = [&]() {  // Gaussian i's record; row and column of its instance rg_
          g = sid[i];
          cnt = (int)(soff[i + 1] - soff[i]);
          ok = g >= 0 && g < cap_n;
          rows = 0;
          if (ok) {
            // the span words are loaded with the rectangle (not after it:
            // one memory latency per Gaussian, not two)
            x0 = __ldg(rect + 4 * g);
            y0 = __ldg(rect + 4 * g + 1);
            const int x1 = __ldg(rect + 4 * g + 2), y1 = __ldg(rect + 4 * g + 3);
            wa = __ldg(reinterpret_cast<const uint4*>(foot + kFootVec * g + 1));
            wb = __ldg(reinterpret_cast<const uint4*>(foot + kFootVec * g + 2));
            rows = y1 - y0;
            if (!fp_packed(rows, x1 - x0)) {
              unpacked = true;
              rows = 0;
            }
          }
          j = 0;
          c = rg_;
          span_at(wa, wb, 0, off, len);
          while (j < rows && c >= len) {
            c -= len;
            if (++j < rows) span_at(wa, wb, j, off, len);
          }
        };
        load();
        for (int e = q0; e < q1; ++e) {
          uint32_t key = 0u;  // valid indices should the spans disagree with ntiles
          int32_t val = 0;
          if (ok) {
            key = j < rows ? (uint32_t)((y0 + j) * TX + x0 + off + c) : (uint32_t)(y0 * TX + x0);
            val = g;
          }
          rtile[e - (int)e0] = key;
          rg[e - (int)e0] = val;
          if (e + 1 == q1) break;
          if (++rg_ < cnt) {  // next instance of this Gaussian: next column, or next row with tiles
            if (++c >= len && j < rows) {
              c = 0;
              while (++j < rows) {
                span_at(wa, wb, j, off, len);
                if (len > 0) break;
              }
            }
          } else {  // next Gaussian with instances
            do {
              ++i;
            } while (i < L - 1 && soff[i + 1] == soff[i]);
            i = min(i, L - 1);  // (the offsets place instance e + 1 within the range)
            rg_ = 0;
            load();
          }
        }
      }
      if (__syncthreads_or(unpacked)) {
        // (the row-parallel path below rewrites the whole range)
      } else {
        for (int e = (int)e0 + t; e < e1; e += 256) {
          tile_keys[e] = rtile[e - (int)e0];
          tile_vals[e] = rg[e - (int)e0];
        }
        return;
      }
      const uint32_t base0 = soff[0];
      __syncthreads();
      uint32_t* srow = soff;  // rows per Gaussian, then their prefix sums
      for (int i = t; i < L; i += 256) {
        const int g = sid[i];
        int rows = 0;
        if (g >= 0 && g < cap_n) rows = max(__ldg(rect + 4 * g + 3) - __ldg(rect + 4 * g + 1), 0);
        srow[i] = (uint32_t)rows;
      }
      __syncthreads();
      const uint32_t R = cta_excl_scan2048(srow, L, wsum);
      if (R <= (uint32_t)kExpandRows) {  // CTA-uniform
        for (int r = t; r < (int)R; r += 256) {
          const int i = last_le(srow, 0, L - 1, (uint32_t)r);
          const int g = sid[i];
          const int x0 = __ldg(rect + 4 * g), y0 = __ldg(rect + 4 * g + 1), x1 = __ldg(rect + 4 * g + 2);
          const int ty = y0 + (r - (int)srow[i]);
          const float2 m = mean2d[g];
          const float4 f = foot[kFootVec * g];
          int t0 = x0, t1 = x0;
          if (f.w >= 0.0f)
            fp_row_span(fp_rows(f.x, f.y, f.z, f.w), m.x, m.y, f.z, f.w, ty, x0, x1, t0, t1);
          rstart[r] = (uint32_t)(t1 - t0);
          rtile[r] = (uint32_t)(ty * TX + t0);
          rg[r] = g;
        }
        __syncthreads();
        const uint32_t total = cta_excl_scan2048(rstart, (int)R, wsum);
        // each row writes its instances that fall in [e0, e1); consecutive
        // rows of a warp cover consecutive instances
        const uint32_t lo = (uint32_t)e0 - base0, hi = (uint32_t)e1 - base0;
        for (int r = t; r < (int)R; r += 256) {
          const uint32_t a0 = max(rstart[r], lo), a1 = min(rstart[r + 1], hi);
          const uint32_t key0 = rtile[r] - rstart[r];
          const int32_t g = rg[r];
          for (uint32_t k = a0; k < a1; ++k) {
            tile_keys[base0 + k] = key0 + k;
            tile_vals[base0 + k] = g;
          }
        }
        // instances the spans do not reach (only if they disagree with
        // ntiles): valid indices
        for (uint32_t k = max(total, lo) + t; k < hi; k += 256) {
          tile_keys[base0 + k] = 0u;
          tile_vals[base0 + k] = 0;
        }
        return;
      }
    }
    // very wide ranges (more Gaussians or rows than the CTA caches): one
    // thread per Gaussian walks its rows and writes its instances in [e0, e1)
    for (int j = jlo + t; j <= jhi; j += 256) {
      const int g = order[j];
      const int base = (int)off[j], end = (int)off[j + 1];
      const int lo = base > (int)e0 ? base : (int)e0, hi = end < e1 ? end : e1;
      if (lo >= hi) continue;
      int key = 0, gg = 0, k = base;
      if (g >= 0 && g < cap_n) {
        const int x0 = __ldg(rect + 4 * g), y0 = __ldg(rect + 4 * g + 1), x1 = __ldg(rect + 4 * g + 2),
                  y1 = __ldg(rect + 4 * g + 3);
        const float2 m = mean2d[g];
        const float4 f = foot[kFootVec * g];
        gg = g;
        key = y0 * TX + x0;
        if (f.w >= 0.0f) {
          const FootRows fr = fp_rows(f.x, f.y, f.z, f.w);
          for (int ty = y0; ty < y1 && k < hi; ++ty) {
            int t0, t1;
            fp_row_span(fr, m.x, m.y, f.z, f.w, ty, x0, x1, t0, t1);
            int tx = t0;
            if (k < lo) {
              const int skip = lo - k < t1 - t0 ? lo - k : t1 - t0;
              tx += skip;
              k += skip;
            }
            for (; tx < t1 && k < hi; ++tx, ++k) {
              tile_keys[k] = (uint32_t)(ty * TX + tx);
              tile_vals[k] = g;
            }
          }
        }
      }
      for (k = k > lo ? k : lo; k < hi; ++k) {
        tile_keys[k] = (uint32_t)key;
        tile_vals[k] = gg;
      }
    }
    return;
  }
  for (int e = (int)e0 + t; e < e1; e += 256) {
    int g, r;
    if (cached) {
      const int i = last_le(soff, 0, L - 1, (uint32_t)e);
      g = sid[i];
      r = e - (int)soff[i];
    } else {
      const int j = last_le(off, jlo, jhi, (uint32_t)e);
      g = order[j];
      r = e - (int)off[j];
    }
    if (g < 0 || g >= cap_n) continue;
    const int x0 = __ldg(rect + 4 * g), y0 = __ldg(rect + 4 * g + 1), x1 = __ldg(rect + 4 * g + 2);
    const int wdt = x1 - x0;
    if (wdt <= 0) continue;  // rect inconsistent with ntiles: nothing sensible to emit
    tile_keys[e] = (uint32_t)((y0 + r / wdt) * TX + x0 + r % wdt);
    tile_vals[e] = g;
  }
}

__global__ void __launch_bounds__(256) k_ranges(const uint32_t* __restrict__ tile_keys,
                                                const int32_t* __restrict__ n_ptr, int cap,
                                                int n_tiles, int32_t* __restrict__ ranges) {
  const int K = clamp_n(n_ptr, cap);
  constexpr uint32_t kNone = 0xffffffffu;  // outside [0, K): differs from every tile
  // four consecutive keys per thread (one 16-byte load; the workspace is
  // 256-byte aligned) and their two neighbours
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; 4 * q < K; q += gridDim.x * blockDim.x) {
    const int k0 = 4 * q;
    uint32_t v[6];
    if (k0 + 4 <= K) {
      const uint4 u = *reinterpret_cast<const uint4*>(tile_keys + k0);
      v[1] = u.x;
      v[2] = u.y;
      v[3] = u.z;
      v[4] = u.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[1 + j] = k0 + j < K ? tile_keys[k0 + j] : kNone;
    }
    v[0] = k0 > 0 ? tile_keys[k0 - 1] : kNone;
    v[5] = k0 + 4 < K ? tile_keys[k0 + 4] : kNone;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint32_t t = v[1 + j];
      if (k0 + j >= K || t >= (uint32_t)n_tiles) continue;
      if (v[j] != t) ranges[2 * t] = k0 + j;
      if (v[j + 2] != t) ranges[2 * t + 1] = k0 + j + 1;
    }
  }
}

__global__ void __launch_bounds__(256) k_keys64(const uint32_t* __restrict__ tile_keys,
                                                const int32_t* __restrict__ vals,
                                                const float* __restrict__ depth,
                                                const int32_t* __restrict__ n_ptr, int cap,
                                                uint64_t* __restrict__ keys) {
  const int K = clamp_n(n_ptr, cap);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
    keys[k] = ((uint64_t)tile_keys[k] << 32) | (uint64_t)__float_as_uint(depth[vals[k]]);
}

__global__ void __launch_bounds__(256) k_depth_keys(const float* __restrict__ depth,
                                                    const int32_t* __restrict__ n_ptr, int cap,
                                                    uint32_t* __restrict__ keys,
                                                    int32_t* __restrict__ vals) {
  const int n = clamp_n(n_ptr, cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    keys[i] = __float_as_uint(depth[i]);
    vals[i] = i;
  }
}

// ---------------------------------------------------------------- host side

static int radix_ctas(int64_t cap) {
  int64_t g = (cap + HYRF_RADIX_PER_CTA - 1) / HYRF_RADIX_PER_CTA;
  return (int)(g < 1 ? 1 : (g > kMaxRadixCTAs ? kMaxRadixCTAs : g));
}

static int bits_for(int64_t n_values) {
  int b = 0;
  while ((1ll << b) < n_values) ++b;
  return b < 1 ? 1 : b;
}

struct SortWs {
  uint32_t *dk_a, *dk_b, *tk_a, *tk_b;
  int32_t *dv_a, *dv_b, *tv_b;
  uint32_t *hist, *totals;
  int64_t* sums;
  uint32_t* off;
};

static SortWs carve_sort(Carver& c, int n, int64_t cap) {
  SortWs w;
  const int Gd = radix_ctas(n), Gt = radix_ctas(cap);
  const int G = Gd > Gt ? Gd : Gt;
  w.dk_a = c.take<uint32_t>(n);
  w.dk_b = c.take<uint32_t>(n);
  w.dv_a = c.take<int32_t>(n);
  w.dv_b = c.take<int32_t>(n);
  w.tk_a = c.take<uint32_t>(cap);
  w.tk_b = c.take<uint32_t>(cap);
  w.tv_b = c.take<int32_t>(cap);
  w.hist = c.take<uint32_t>((size_t)256 * G);
  w.totals = c.take<uint32_t>(256);
  w.sums = c.take<int64_t>((n + kScanChunk - 1) / kScanChunk + 1);
  w.off = c.take<uint32_t>((size_t)n + 1);
  return w;
}

size_t bin_sort_workspace(int n, int64_t cap) {
  Carver c(nullptr);
  carve_sort(c, n, cap);
  return c.size();
}



// Stable LSD radix sort of (keys, vals) on bits [0, nbits); the result ends in
// (ka, va); (kb, vb) is scratch. The input must be in (ka, va) when the pass
// count is even and in (kb, vb) when it is odd.
static hyrf_status radix_sort(uint32_t* ka, int32_t* va, uint32_t* kb, int32_t* vb,
                              const int32_t* n_ptr, int cap, int nbits, uint32_t* hist,
                              uint32_t* totals, cudaStream_t s, const char* name = "k_radix_scatter") {
  const int G = radix_ctas(cap);
  const int passes = (nbits + 7) / 8;
  uint32_t* src_k = (passes & 1) ? kb : ka;
  int32_t* src_v = (passes & 1) ? vb : va;
  uint32_t* dst_k = (passes & 1) ? ka : kb;
  int32_t* dst_v = (passes & 1) ? va : vb;
  // the bits split evenly over the passes (12 tile bits: 6 + 6, so that
  // each digit's run in a sub-tile is long enough for coalesced writes)
  const int per = (nbits + passes - 1) / passes;
  for (int p = 0; p < passes; ++p) {
    const int shift = per * p;
    const int bits = nbits - shift < per ? nbits - shift : per;
    const uint32_t mask = (1u << bits) - 1u;
    HYRF_LAUNCH("k_radix_hist", s,
                k_radix_hist<<<G, kRT, 0, s>>>(src_k, n_ptr, cap, shift, mask, hist));
    HYRF_LAUNCH("k_radix_colscan", s,
                k_radix_colscan<<<(int)mask + 1, kRT, 0, s>>>(hist, G, totals));
    HYRF_LAUNCH(name, s,
                k_radix_scatter<<<G, kRT, 0, s>>>(src_k, src_v, dst_k, dst_v, n_ptr, cap, shift, mask, hist,
                                      totals));
    uint32_t* tk = src_k;
    src_k = dst_k;
    dst_k = tk;
    int32_t* tv = src_v;
    src_v = dst_v;
    dst_v = tv;
  }
  return HYRF_OK;
}

hyrf_status launch_bin_sort(const hyrf_bin_sort_args& a, void* ws, cudaStream_t s) {
  const int n = a.n;
  const int64_t cap = a.capacity;
  const int n_tiles = a.tiles_x * a.tiles_y;
  Carver c(ws);
  SortWs w = carve_sort(c, n, cap);
  cudaMemsetAsync(a.ranges, 0, (size_t)n_tiles * 2 * sizeof(int32_t), s);
  if (n == 0 || cap == 0) {
    cudaMemsetAsync(a.n_instances, 0, sizeof(int32_t), s);
    return cudaPeekAtLastError() == cudaSuccess ? HYRF_OK : HYRF_ERR_CUDA;
  }
  // 1. depth keys of the visible Gaussians, sorted (4 x 8 bits), unless the
  // caller ordered them already (hyrf_depth_order)
  hyrf_status st = HYRF_OK;
  const int32_t* ord = a.depth_order;
  if (!ord) {
    const int eb = (n + 255) / 256 < num_sms() * 8 ? (n + 255) / 256 : num_sms() * 8;
    HYRF_LAUNCH("k_depth_keys", s,
                k_depth_keys<<<eb, 256, 0, s>>>(a.depth, a.n_vis, n, w.dk_a, w.dv_a));
    st = radix_sort(w.dk_a, w.dv_a, w.dk_b, w.dv_b, a.n_vis, n, 32, w.hist, w.totals, s,
                    "k_radix_scatter<depth>");
    if (st != HYRF_OK) return st;
    ord = w.dv_a;
  }
  // 2. instance offsets in depth order, K, and emission
  const int sc = (n + kScanChunk - 1) / kScanChunk;
  HYRF_LAUNCH("k_count_sums", s,
              k_count_sums<<<sc, 256, 0, s>>>(a.ntiles, ord, a.n_vis, n, w.sums));
  HYRF_LAUNCH("k_scan_sums", s,
              k_scan_sums<<<1, 1024, 0, s>>>(w.sums, sc, cap, a.n_instances, a.status));
  const int tbits = bits_for(n_tiles);
  const int tpasses = (tbits + 7) / 8;
  uint32_t* emit_k = (tpasses & 1) ? w.tk_b : w.tk_a;
  int32_t* emit_v = (tpasses & 1) ? w.tv_b : a.vals;
  HYRF_LAUNCH("k_offsets", s,
              k_offsets<<<sc, 256, 0, s>>>(a.ntiles, ord, a.n_vis, n, w.sums, sc, w.off));
  const int capi = (int)(cap < 0x7fffffff ? cap : 0x7fffffff);
  const int64_t xb = (cap + kExpandItems - 1) / kExpandItems;
  HYRF_LAUNCH("k_expand", s,
              k_expand<<<(int)(xb < 0x7fffffff ? xb : 0x7fffffff), 256, 0, s>>>(
                  a.rect, ord, a.n_vis, n, w.off, a.n_instances, capi, a.tiles_x, emit_k, emit_v,
                  reinterpret_cast<const float2*>(a.mean2d), reinterpret_cast<const float4*>(a.footprint)));
  // 3. stable sort of the instances on their tile bits
  st = radix_sort(w.tk_a, a.vals, w.tk_b, w.tv_b, a.n_instances, capi, tbits, w.hist, w.totals, s,
                  "k_radix_scatter<tile>");
  if (st != HYRF_OK) return st;
  // 4. per-tile ranges and (optionally) the composed 64-bit keys
  const int kb = (int)((cap + 255) / 256 < num_sms() * 8 ? (cap + 255) / 256 : num_sms() * 8);
  const int rb = (int)((cap + 1023) / 1024 < num_sms() * 8 ? (cap + 1023) / 1024 : num_sms() * 8);
  HYRF_LAUNCH("k_ranges", s,
              k_ranges<<<rb, 256, 0, s>>>(w.tk_a, a.n_instances, capi, n_tiles, a.ranges));
  if (a.keys) {
    HYRF_LAUNCH("k_keys64", s,
                k_keys64<<<kb, 256, 0, s>>>(w.tk_a, a.vals, a.depth, a.n_instances, capi, a.keys));
  }
  return HYRF_OK;
}

// ---------------------------------------------------------------- depth order alone

hyrf_status launch_depth_of(const CamDev& cam, int n, const float* pos, const int32_t* vis_ids,
                            const int32_t* n_vis, float* depth, int32_t* status, cudaStream_t s);

struct DepthWs {
  float* depth;
  uint32_t *k_a, *k_b;
  int32_t* v_b;
  uint32_t *hist, *totals;
};

static DepthWs carve_depth(Carver& c, int n) {
  DepthWs w;
  const int m = n > 0 ? n : 1;
  w.depth = c.take<float>(m);
  w.k_a = c.take<uint32_t>(m);
  w.k_b = c.take<uint32_t>(m);
  w.v_b = c.take<int32_t>(m);
  w.hist = c.take<uint32_t>((size_t)256 * radix_ctas(m));
  w.totals = c.take<uint32_t>(256);
  return w;
}

size_t depth_order_workspace(int n) {
  Carver c(nullptr);
  carve_depth(c, n);
  return c.size();
}

// The depth keys and the four 8-bit passes of launch_bin_sort's step 1, on
// depths computed from the positions (the same FP32 z as the projection).
hyrf_status launch_depth_order(const hyrf_depth_order_args& a, void* ws, cudaStream_t s) {
  const int n = a.n;
  if (n == 0) return HYRF_OK;
  Carver c(ws);
  DepthWs w = carve_depth(c, n);
  hyrf_status st = launch_depth_of(to_dev(a.cam), n, a.pos, a.vis_ids, a.n_vis, w.depth, a.status, s);
  if (st != HYRF_OK) return st;
  const int eb = (n + 255) / 256 < num_sms() * 8 ? (n + 255) / 256 : num_sms() * 8;
  HYRF_LAUNCH("k_depth_keys", s, k_depth_keys<<<eb, 256, 0, s>>>(w.depth, a.n_vis, n, w.k_a, a.order));
  return radix_sort(w.k_a, a.order, w.k_b, w.v_b, a.n_vis, n, 32, w.hist, w.totals, s,
                    "k_radix_scatter<depth>");
}

// ---------------------------------------------------------------- storage order

__device__ __forceinline__ uint32_t spread10(uint32_t v) {  // bit i -> bit 3i
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Morton code of the contracted position (App. A.1 normalisation, Eq. 2
// with the +0.5 offset), 10 bits per axis; vals = identity.
__global__ void __launch_bounds__(256) k_morton(int n, const float* __restrict__ pos, float3 lo, float3 sx,
                                                uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float x[3] = {(pos[3 * (int64_t)i] - lo.x) * sx.x - 1.0f, (pos[3 * (int64_t)i + 1] - lo.y) * sx.y - 1.0f,
                        (pos[3 * (int64_t)i + 2] - lo.z) * sx.z - 1.0f};
    const float r = sqrtf(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    const float g = r <= 1.0f ? 1.0f : (2.0f - 1.0f / r) / r;
    uint32_t q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float y = 0.25f * g * x[k] + 0.5f;
      q[k] = (uint32_t)fminf(fmaxf(y * 1024.0f, 0.0f), 1023.0f);
    }
    keys[i] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
    vals[i] = i;
  }
}

__global__ void k_set_count(int32_t* c, int n) { *c = n; }

struct PermuteArgs {
  hyrf_remap_array a[HYRF_REMAP_MAX];
  int count;
};

__global__ void __launch_bounds__(256) k_permute_rows(const int32_t* __restrict__ perm, int n, PermuteArgs P) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int64_t g = perm[k];
    if (g < 0 || g >= n) continue;
    for (int j = 0; j < P.count; ++j) {
      const hyrf_remap_array& A = P.a[j];
      for (int c = 0; c < A.width; ++c) A.dst[(int64_t)k * A.width + c] = A.src[g * A.width + c];
    }
  }
}

static size_t order_ws(int n, Carver& c, uint32_t** ka, uint32_t** kb, int32_t** vb, uint32_t** hist,
                       uint32_t** totals) {
  *ka = c.take<uint32_t>(n);
  *kb = c.take<uint32_t>(n);
  *vb = c.take<int32_t>(n);
  *hist = c.take<uint32_t>((size_t)256 * radix_ctas(n));
  *totals = c.take<uint32_t>(256);
  c.take<int32_t>(1);  // device count
  return c.size();
}

}  // namespace hyrf

using namespace hyrf;

extern "C" size_t hyrf_spatial_order_workspace_size(const hyrf_spatial_order_args* a) {
  if (!a || a->n < 0) return 0;
  Carver c(nullptr);
  uint32_t *ka, *kb, *h, *t;
  int32_t* vb;
  return order_ws(a->n, c, &ka, &kb, &vb, &h, &t);
}

extern "C" hyrf_status hyrf_spatial_order(const hyrf_spatial_order_args* a, void* ws, size_t ws_bytes,
                                          void* stream) {
  if (!a || a->n < 0) return HYRF_ERR_INVALID_ARG;
  if (a->n == 0) return HYRF_OK;
  if (!a->pos || !a->perm || !ws || ws_bytes < hyrf_spatial_order_workspace_size(a)) return HYRF_ERR_INVALID_ARG;
  float sx[3];
  for (int k = 0; k < 3; ++k) {
    const float e = a->box_hi[k] - a->box_lo[k];
    if (!(e > 0.0f)) return HYRF_ERR_INVALID_ARG;
    sx[k] = 2.0f / e;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  Carver c(ws);
  uint32_t *ka, *kb, *hist, *totals;
  int32_t* vb;
  order_ws(a->n, c, &ka, &kb, &vb, &hist, &totals);
  // the device count the radix passes read sits at the end of the workspace
  int32_t* count = reinterpret_cast<int32_t*>(static_cast<char*>(ws) + c.size() - 256);
  HYRF_LAUNCH("k_set_count", s, k_set_count<<<1, 1, 0, s>>>(count, a->n));
  int blocks = (a->n + 255) / 256;
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  HYRF_LAUNCH("k_morton", s,
              k_morton<<<blocks, 256, 0, s>>>(a->n, a->pos, make_float3(a->box_lo[0], a->box_lo[1], a->box_lo[2]),
                                               make_float3(sx[0], sx[1], sx[2]), ka, a->perm));
  return radix_sort(ka, a->perm, kb, vb, count, a->n, 30, hist, totals, s);
}

extern "C" hyrf_status hyrf_permute_rows(const int32_t* perm, int32_t n, const hyrf_remap_array* arrays,
                                         int32_t count, void* stream) {
  if (n < 0 || count < 0 || count > HYRF_REMAP_MAX || (n > 0 && !perm) || (count > 0 && !arrays))
    return HYRF_ERR_INVALID_ARG;
  PermuteArgs P{};
  for (int j = 0; j < count; ++j) {
    if (!arrays[j].src || !arrays[j].dst || arrays[j].width < 1 || arrays[j].width > 4 || arrays[j].src == arrays[j].dst)
      return HYRF_ERR_INVALID_ARG;
    P.a[j] = arrays[j];
  }
  P.count = count;
  if (n == 0 || count == 0) return HYRF_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int blocks = (n + 255) / 256;
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  HYRF_LAUNCH("k_permute_rows", s, k_permute_rows<<<blocks, 256, 0, s>>>(perm, n, P));
  return HYRF_OK;
}
