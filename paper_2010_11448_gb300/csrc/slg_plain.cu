// The plain per-hyperedge GPU kernel (SLG_ALGO_PLAIN): Algorithm 3 carried
// over to the GPU as directly as possible, kept as the comparison point for
// the binned walk.
//
//  * one warp per hyperedge, rows dealt cyclically to the warps (the cyclic
//    range of Section IV-F);
//  * the unfiltered CSC, with Algorithm 3's checks per wedge: f > e (strict
//    upper triangle) and |f| >= s (degree-based pruning); |e| >= s per row;
//  * a dense per-warp count array in global memory (Algorithm 3's per-thread
//    visited array, holding counts) plus a per-warp bitmap in global memory
//    with one bit per 32 counters, scanned in order to emit sorted rows;
//  * two passes: count, then (after the scan of the per-row counts) write
//    each row to its final place.
#include "slg_internal.cuh"

namespace slg {

namespace {

constexpr int kPlainNT = 256;

// COUNT: record the row's pair count; DIRECT: the row's output offset.
__device__ __forceinline__ long long reserve_plain(const EmitArgs &a, int32_t e, int32_t n) {
  const int32_t r = e - a.row_begin;
  if (a.mode == kCount) {
    a.n_e[r] = n;
    if (n) atomicAdd(&a.meta->pairs_bin[0], (unsigned long long)n);
    return -1;
  }
  return a.row_ptr[r];
}

__global__ __launch_bounds__(kPlainNT) void k_plain(Side sd, int32_t smin, int32_t row_begin,
                                                    int32_t row_end, EmitArgs a,
                                                    int32_t *__restrict__ scratch,
                                                    uint32_t *__restrict__ summ, int32_t R_pad) {
  Meta *meta = a.meta;
  if (meta->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kPlainNT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kPlainNT) >> 5;
  const int32_t nsw = R_pad >> 10;
  int32_t *cnt = scratch + gw * (int64_t)R_pad;   // zero between rows
  uint32_t *sm = summ + gw * (int64_t)nsw;        // zero between rows
  const bool unweighted = a.unweighted != 0;
  unsigned long long wedges = 0;
  for (int64_t e = row_begin + gw; e < row_end; e += nw) {
    const int32_t lo = sd.r_off[e], hi = sd.r_off[e + 1];
    if (hi - lo < smin) {
      if (lane == 0) reserve_plain(a, (int32_t)e, 0);
      continue;
    }
    for (int32_t k = lo; k < hi; ++k) {
      const int32_t v = __ldg(sd.r_idx + k);
      const int32_t cb = __ldg(sd.c_off + v), ce = __ldg(sd.c_off + v + 1);
      for (int32_t q = cb + lane; q < ce; q += 32) {
        const int32_t f = __ldg(sd.c_idx + q);
        if (f <= e) continue;
        if (__ldg(sd.r_off + f + 1) - __ldg(sd.r_off + f) < smin) continue;
        ++wedges;
        if (unweighted && __ldcg(cnt + f) >= smin) continue;
        if (atomicAdd(cnt + f, 1) == 0) atomicOr(sm + (f >> 10), 1u << ((f >> 5) & 31));
      }
    }
    __threadfence_block();
    __syncwarp();
    // pass over the bitmap in order: lane owns words w0 + lane of each batch
    long long base = -1;
    int32_t n = 0;
    for (int rep = 0; rep < 2; ++rep) {
      if (rep == 1) {
        if (lane == 0) base = reserve_plain(a, (int32_t)e, n);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (a.mode == kCount || base < 0) break;
      }
      int32_t t = 0;
      for (int32_t w0 = 0; w0 < nsw; w0 += 32) {
        const int32_t sw = w0 + lane;
        const uint32_t bits = sw < nsw ? __ldcg(sm + sw) : 0u;
        int32_t c = 0;
        for (uint32_t b = bits; b; b &= b - 1) {
          const int4 *p = reinterpret_cast<const int4 *>(cnt + ((sw << 10) | ((__ffs(b) - 1) << 5)));
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int4 x = __ldcg(p + q);
            c += (x.x >= smin) + (x.y >= smin) + (x.z >= smin) + (x.w >= smin);
          }
        }
        const int32_t inc = warp_inclusive_scan(c);
        if (rep == 0) {
          t += __shfl_sync(0xffffffffu, inc, 31);
          continue;
        }
        int32_t pos = t + inc - c;
        for (uint32_t b = bits; b; b &= b - 1) {
          const int32_t f0 = (sw << 10) | ((__ffs(b) - 1) << 5);
          int4 *p = reinterpret_cast<int4 *>(cnt + f0);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int4 x = __ldcg(p + q);
            const int vals[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (vals[u] >= smin) {
                const int64_t o = base + pos++;
                if (a.out_i) a.out_i[o] = (int32_t)e;
                a.out_j[o] = f0 + 4 * q + u;
                if (!unweighted) a.out_w[o] = vals[u];
              }
          }
        }
        t += __shfl_sync(0xffffffffu, inc, 31);
      }
      if (rep == 0) n = t;
    }
    // restore the zeros: counters of every touched group, then the bitmap
    for (int32_t w0 = 0; w0 < nsw; w0 += 32) {
      const int32_t sw = w0 + lane;
      if (sw >= nsw) continue;
      const uint32_t bits = __ldcg(sm + sw);
      for (uint32_t b = bits; b; b &= b - 1) {
        int4 *p = reinterpret_cast<int4 *>(cnt + ((sw << 10) | ((__ffs(b) - 1) << 5)));
#pragma unroll
        for (int q = 0; q < 8; ++q) __stcg(p + q, make_int4(0, 0, 0, 0));
      }
      if (bits) __stcg(sm + sw, 0u);
    }
    __threadfence_block();
    __syncwarp();
  }
  // wedge total of the count pass (Algorithm 3 visits exactly W_s wedges)
  if (a.mode == kCount) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) wedges += __shfl_xor_sync(0xffffffffu, wedges, d);
    if (lane == 0 && wedges) atomicAdd(&meta->wedges, wedges);
  }
}

}  // namespace

cudaError_t launch_plain(const Side &sd, int32_t smin, int32_t row_begin, int32_t row_end,
                         const EmitArgs &a, int32_t *scratch, uint32_t *summ, int32_t R_pad,
                         int32_t warps, cudaStream_t st) {
  const int grid = (warps * 32 + kPlainNT - 1) / kPlainNT;
  k_plain<<<grid, kPlainNT, 0, st>>>(sd, smin, row_begin, row_end, a, scratch, summ, R_pad);
  return cudaGetLastError();
}

}  // namespace slg
