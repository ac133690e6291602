// The s-overlap walk (Section IV-B/C): for every active row e, count the
// wedges e -> v -> f with f > e per far end f, keep the f with count >= s and
// emit them in ascending f.  The count of f after the walk is |e ∩ f|
// exactly, because each vertex of e contributes one wedge to f when f
// contains it.  Rows are binned by their wedge work:
//
//   warp bin   (work <= 128):   a warp gathers the row's wedge ends in shared
//                               memory, sorts them and counts runs;
//   CTA bins   (work <= 8192):  a CTA counts in a shared-memory open-
//                               addressing table holding twice the row's work
//                               (it can never fill), then sorts the surviving
//                               pairs in shared memory;
//   giant bin  (work > 8192):   a CTA counts in a dense per-CTA array in
//                               global memory (the paper's per-thread visited
//                               array, holding counts) and marks touched
//                               groups of 32 counters in a shared bitmap;
//                               scanning the bitmap in order emits sorted.
//
// Output modes: COUNT (pairs per row only), STAGE (each row's sorted pairs
// are appended to a staging area at an atomically reserved offset) and
// DIRECT (written to their final place, row_ptr known).
#include "slg_internal.cuh"

namespace slg {

// Reserve the output slots of one row; returns the base (or -1: no room).
__device__ __forceinline__ long long reserve(const EmitArgs &a, int32_t e, int32_t n, int bin) {
  const int32_t r = e - a.row_begin;
  a.n_e[r] = n;
  if (n) atomicAdd(&a.meta->pairs_bin[bin], (unsigned long long)n);
  if (a.mode == kCount) return -1;
  if (a.mode == kDirect) return a.row_ptr[r];
  if (n == 0) return -1;
  long long base = (long long)atomicAdd(&a.meta->stage_cursor, (unsigned long long)n);
  if (base + n > a.stage_cap) {
    atomicAdd(&a.meta->stage_overflow, 1ull);
    base = -1;
  }
  a.stage_pos[r] = base;
  return base;
}

__device__ __forceinline__ void put(const EmitArgs &a, long long base, int32_t t, int32_t e,
                                    int32_t f, int32_t c) {
  if (a.mode == kDirect) {
    a.out_i[base + t] = e;
    a.out_j[base + t] = f;
    if (!a.unweighted) a.out_w[base + t] = c;
  } else {
    a.stage_j[base + t] = f;
    if (!a.unweighted) a.stage_w[base + t] = c;
  }
}

// ------------------------------------------------------------- warp bin --

constexpr int kWarpNT = 256;
constexpr int kWarpBuf = kWarpMaxWork;  // 128 ints per warp

__global__ __launch_bounds__(kWarpNT) void k_walk_warp(Walk w, const int32_t *__restrict__ rows,
                                                       EmitArgs a) {
  const Meta *meta = a.meta;
  if (meta->err) return;
  __shared__ int32_t s_buf[kWarpNT / 32][kWarpBuf];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int32_t *buf = s_buf[wib];
  const long long nrows = (long long)meta->rows_bin[kBinWarp];
  const long long gw = ((long long)blockIdx.x * kWarpNT + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * kWarpNT) >> 5;
  for (long long r = gw; r < nrows; r += nw) {
    const int32_t e = rows[r];
    const int32_t k0 = w.r_off[e], k1 = w.r_off[e + 1];
    // 1. gather the wedge ends (row work <= kWarpBuf by binning)
    int32_t filled = 0;
    for (int32_t base = k0; base < k1; base += 32) {
      const int32_t k = base + lane;
      int32_t b = 0, len = 0;
      if (k < k1) {
        const int32_t v = __ldg(w.r_idx + k);
        b = __ldg(w.tail_beg + k);
        len = __ldg(w.c_off_s + v + 1) - b;
      }
      const int32_t inc = warp_inclusive_scan(len);
      const int32_t total = __shfl_sync(0xffffffffu, inc, 31);
      for (int32_t i0 = 0; i0 < total; i0 += 32) {
        const int32_t i = i0 + lane;
        int32_t j = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int32_t cand = j + step;
          if (__shfl_sync(0xffffffffu, inc, cand - 1) <= i) j = cand;
        }
        const int32_t seg_inc = __shfl_sync(0xffffffffu, inc, j);
        const int32_t seg_len = __shfl_sync(0xffffffffu, len, j);
        const int32_t seg_beg = __shfl_sync(0xffffffffu, b, j);
        if (i < total && filled + i < kWarpBuf)
          buf[filled + i] = __ldg(w.c_idx_s + seg_beg + (i - (seg_inc - seg_len)));
      }
      filled += total;
    }
    const int32_t n = filled < kWarpBuf ? filled : kWarpBuf;
    // 2. bitonic sort of the n ends, padded to a power of two
    int32_t n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int32_t i = n + lane; i < n2; i += 32) buf[i] = 0x7fffffff;
    __syncwarp();
    for (int32_t k = 2; k <= n2; k <<= 1) {
      for (int32_t jj = k >> 1; jj > 0; jj >>= 1) {
        for (int32_t i = lane; i < n2; i += 32) {
          const int32_t ixj = i ^ jj;
          if (ixj > i) {
            const int32_t x = buf[i], y = buf[ixj];
            const bool up = (i & k) == 0;
            if ((x > y) == up) {
              buf[i] = y;
              buf[ixj] = x;
            }
          }
        }
        __syncwarp();
      }
    }
    // 3. run starts with run length >= s, kept in order
    int32_t cnt_total = 0;
    for (int32_t p0 = 0; p0 < n; p0 += 32) {
      const int32_t p = p0 + lane;
      bool q = false;
      if (p < n && (p == 0 || buf[p - 1] != buf[p])) {
        int32_t end = p + 1;
        while (end < n && buf[end] == buf[p]) ++end;
        q = (end - p) >= a.smin;
      }
      cnt_total += __popc(__ballot_sync(0xffffffffu, q));
    }
    long long base = -1;
    if (lane == 0) base = reserve(a, e, cnt_total, kBinWarp);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (a.mode != kCount && base >= 0) {
      int32_t t0 = 0;
      for (int32_t p0 = 0; p0 < n; p0 += 32) {
        const int32_t p = p0 + lane;
        bool q = false;
        int32_t c = 0;
        if (p < n && (p == 0 || buf[p - 1] != buf[p])) {
          int32_t end = p + 1;
          while (end < n && buf[end] == buf[p]) ++end;
          c = end - p;
          q = c >= a.smin;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, q);
        if (q) put(a, base, t0 + __popc(bal & ((1u << lane) - 1)), e, buf[p], c);
        t0 += __popc(bal);
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------- shared-memory tables --
//
// An open-addressing table of T = 2^lgT slots (keys = far ends f, cnts =
// wedge counts) in shared memory, T >= 2 x (distinct keys) so it never fills.
// After the walk, table_collect counts the slots with count >= s and, if
// asked, packs them as (f << 32 | count) into the first entries of the keys
// array (reused as a u64 buffer: at most T/2 entries) and sorts them by f.

__device__ __forceinline__ void table_insert(int32_t *keys, int32_t *cnts, int lgT, int32_t f,
                                             int32_t add, int32_t smin, bool unweighted,
                                             Meta *meta) {
  const uint32_t mask = (1u << lgT) - 1u;
  uint32_t h = ((uint32_t)f * 0x9E3779B1u) >> (32 - lgT);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    const int32_t k = *(volatile int32_t *)(keys + h);
    if (k == f) {
      if (!unweighted || *(volatile int32_t *)(cnts + h) < smin) atomicAdd(cnts + h, add);
      return;
    }
    if (k == kEmpty) {
      const int32_t prev = atomicCAS(keys + h, kEmpty, f);
      if (prev == kEmpty || prev == f) {
        atomicAdd(cnts + h, add);
        return;
      }
    }
    h = (h + 1) & mask;
  }
  raise_error(meta, SLG_ERR_INVALID, kWhereHash);  // unreachable: T >= 2 x distinct
}

__device__ __forceinline__ int ceil_log2(int32_t x) {
  return x <= 1 ? 0 : 32 - __clz(x - 1);
}

// Table size for a multiset with at most `distinct` keys: 2^lgT >= 2 x distinct.
__device__ __forceinline__ int table_lg(int32_t distinct, int lg_max) {
  int lg = ceil_log2(2 * (distinct > 16 ? distinct : 16));
  return lg < lg_max ? lg : lg_max;
}

template <int NT, int SPT>
__device__ __forceinline__ int32_t table_collect(int32_t *keys, int32_t *cnts, int32_t T,
                                                 int32_t smin, bool sort, int32_t *ws) {
  int32_t kk[SPT], cc[SPT];
  int32_t c = 0;
#pragma unroll
  for (int i = 0; i < SPT; ++i) {
    const int32_t slot = i * NT + (int32_t)threadIdx.x;
    kk[i] = kEmpty;
    cc[i] = 0;
    if (slot < T) {
      kk[i] = keys[slot];
      cc[i] = cnts[slot];
    }
    c += (kk[i] != kEmpty) & (cc[i] >= smin);
  }
  int32_t total;
  const int32_t inc = block_inclusive_scan<NT>(c, ws, &total);  // all slot reads done
  if (sort && total > 0) {
    unsigned long long *sb = reinterpret_cast<unsigned long long *>(keys);
    int32_t pos = inc - c;
#pragma unroll
    for (int i = 0; i < SPT; ++i)
      if (kk[i] != kEmpty && cc[i] >= smin)
        sb[pos++] = ((unsigned long long)(uint32_t)kk[i] << 32) | (uint32_t)cc[i];
    int32_t n2 = 1;
    while (n2 < total) n2 <<= 1;
    for (int32_t i = total + threadIdx.x; i < n2; i += NT) sb[i] = ~0ull;
    __syncthreads();
    for (int32_t k = 2; k <= n2; k <<= 1) {
      for (int32_t jj = k >> 1; jj > 0; jj >>= 1) {
        for (int32_t i = threadIdx.x; i < n2; i += NT) {
          const int32_t ixj = i ^ jj;
          if (ixj > i) {
            const unsigned long long x = sb[i], y = sb[ixj];
            if ((x > y) == ((i & k) == 0)) {
              sb[i] = y;
              sb[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
    }
  }
  return total;
}

template <int NT, int SPT>
__device__ __forceinline__ void table_reset(int32_t *keys, int32_t *cnts, int32_t T) {
  __syncthreads();  // sorted entries may still be read from keys
#pragma unroll
  for (int i = 0; i < SPT; ++i) {
    const int32_t slot = i * NT + (int32_t)threadIdx.x;
    if (slot < T) {
      keys[slot] = kEmpty;
      cnts[slot] = 0;
    }
  }
  __syncthreads();
}

// -------------------------------------------------------------- CTA bins --

template <int NT, int TMAX>
struct CtaCfg {
  static constexpr int kSPT = TMAX / NT;  // slots per thread at most
  // [s_base 16 B][keys TMAX][cnts TMAX][s_beg NT][s_pref NT+1][ws NT/32+1]
  static constexpr size_t smem() {
    return 16 + (size_t)TMAX * 8 + (size_t)(2 * NT + 1 + NT / 32 + 1) * 4;
  }
};

template <int NT, int TMAX, int BIN>
__global__ __launch_bounds__(NT) void k_walk_cta(Walk w, const int32_t *__restrict__ rows,
                                                 const int32_t *__restrict__ row_work,
                                                 EmitArgs a) {
  using Cfg = CtaCfg<NT, TMAX>;
  Meta *meta = a.meta;
  if (meta->err) return;
  extern __shared__ __align__(16) unsigned char smem[];
  long long *s_base = reinterpret_cast<long long *>(smem);
  int32_t *keys = reinterpret_cast<int32_t *>(smem + 16);
  int32_t *cnts = keys + TMAX;
  int32_t *s_beg = cnts + TMAX;
  int32_t *s_pref = s_beg + NT;
  int32_t *ws = s_pref + NT + 1;
  constexpr int lg_max = (TMAX >= 2) ? 31 - __builtin_clz(TMAX) : 1;

  for (int i = threadIdx.x; i < TMAX; i += NT) {
    keys[i] = kEmpty;
    cnts[i] = 0;
  }
  __syncthreads();
  const long long nrows = (long long)meta->rows_bin[BIN];
  const int32_t smin = a.smin;
  const bool unweighted = a.unweighted != 0;
  const bool emit = a.mode != kCount;
  for (long long r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int32_t e = rows[r];
    const int lgT = table_lg(row_work[e - a.row_begin], lg_max);
    const int32_t T = 1 << lgT;
    cta_walk<NT, 4>(w, w.r_off[e], w.r_off[e + 1], s_beg, s_pref, ws, [&](int32_t f) {
      table_insert(keys, cnts, lgT, f, 1, smin, unweighted, meta);
    });
    const int32_t total = table_collect<NT, Cfg::kSPT>(keys, cnts, T, smin, emit, ws);
    if (threadIdx.x == 0) *s_base = reserve(a, e, total, BIN);
    __syncthreads();
    const long long base = *s_base;
    if (emit && base >= 0) {
      const unsigned long long *sb = reinterpret_cast<const unsigned long long *>(keys);
      for (int32_t i = threadIdx.x; i < total; i += NT) {
        const unsigned long long x = sb[i];
        put(a, base, i, e, (int32_t)(x >> 32), (int32_t)(uint32_t)x);
      }
    }
    table_reset<NT, Cfg::kSPT>(keys, cnts, T);
  }
}

// ------------------------------------------------------------- giant bin --
//
// A CTA takes one giant row at a time (dynamic ticket).  The row's far ends
// f lie in [f_lo, R) (f_lo = e + 1 for the upper-triangle walk, 0 for whole
// columns); they are split into NSB sub-ranges of 2^shift ids.
//   1. walk, counting wedges per sub-range (shared histogram);
//   2. exclusive scan; walk again, scattering every f into the CTA's global
//      scratch grouped by sub-range (the scratch of the rows in flight stays
//      in L2);
//   3. consecutive sub-ranges are grouped into buckets of at most CAP wedges
//      (a single larger sub-range forms its own bucket: it holds at most
//      2^shift distinct ids); each bucket, in ascending f, is counted in the
//      shared table, and its pairs (already in order) are appended to the
//      row's output.
// Nothing is counted in global memory and the output comes out sorted.

constexpr int kGiantNT = 1024;
constexpr int kGiantTMax = 16384;
constexpr int kNSB = 4096;  // sub-ranges per row
constexpr int kGiantSPT = kGiantTMax / kGiantNT;

// [s_base 16][s_misc 16][keys TMAX][cnts TMAX][sub NSB][bstart NSB+1]
// [s_beg NT][s_pref NT+1][ws NT/32+1]
constexpr size_t giant_smem() {
  return 32 + (size_t)kGiantTMax * 8 + (size_t)(2 * kNSB + 1) * 4 +
         (size_t)(2 * kGiantNT + 1 + kGiantNT / 32 + 1) * 4;
}

__global__ __launch_bounds__(kGiantNT) void k_walk_giant(Walk w, const int32_t *__restrict__ rows,
                                                         EmitArgs a, int32_t *__restrict__ scratch,
                                                         long long scratch_stride, int32_t R) {
  Meta *meta = a.meta;
  if (meta->err) return;
  extern __shared__ __align__(16) unsigned char smem[];
  long long *s_base = reinterpret_cast<long long *>(smem);
  int32_t *s_misc = reinterpret_cast<int32_t *>(smem + 16);  // [0] row, [1] buckets
  int32_t *keys = reinterpret_cast<int32_t *>(smem + 32);
  int32_t *cnts = keys + kGiantTMax;
  int32_t *sub = cnts + kGiantTMax;
  int32_t *bstart = sub + kNSB;
  int32_t *s_beg = bstart + kNSB + 1;
  int32_t *s_pref = s_beg + kGiantNT;
  int32_t *ws = s_pref + kGiantNT + 1;
  // per-CTA global scratch: wedge ends, then the row's staged pairs (j, w)
  int32_t *wl = scratch + (long long)blockIdx.x * scratch_stride;
  int32_t *tj = wl + scratch_stride / 3;
  int32_t *tw = tj + scratch_stride / 3;

  for (int i = threadIdx.x; i < kGiantTMax; i += kGiantNT) {
    keys[i] = kEmpty;
    cnts[i] = 0;
  }
  const unsigned nrows = (unsigned)meta->rows_bin[kBinGiant];
  const int32_t smin = a.smin;
  const bool unweighted = a.unweighted != 0;
  const bool emit = a.mode != kCount;
  constexpr int lg_max = 31 - __builtin_clz(kGiantTMax);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned t = atomicAdd(&meta->giant_ticket, 1u);
      s_misc[0] = t < nrows ? rows[t] : -1;
    }
    __syncthreads();
    const int32_t e = s_misc[0];
    if (e < 0) break;
    // far ends lie in [f_lo, R): (e, R) for the upper-triangle walk, the
    // whole [0, R) when the tails are whole columns
    const int32_t f_lo = a.full_rows ? 0 : e + 1;
    const int32_t span = R - f_lo;
    const int shift = max(0, ceil_log2(span) - 12);  // kNSB = 2^12
    const int32_t nsb = ((span - 1) >> shift) + 1;
    const int32_t cap = kGiantTMax / 2 - (1 << shift);
    const int32_t k0 = w.r_off[e], k1 = w.r_off[e + 1];
    // 1. histogram of sub-ranges
    for (int i = threadIdx.x; i < kNSB; i += kGiantNT) sub[i] = 0;
    __syncthreads();
    cta_walk<kGiantNT, 4>(w, k0, k1, s_beg, s_pref, ws, [&](int32_t f) {
      atomicAdd(sub + ((f - f_lo) >> shift), 1);
    });
    // 2. exclusive scan (4 sub-ranges per thread), then scatter
    {
      constexpr int P = kNSB / kGiantNT;
      int32_t v[P], t = 0;
#pragma unroll
      for (int q = 0; q < P; ++q) {
        v[q] = sub[threadIdx.x * P + q];
        t += v[q];
      }
      int32_t total;
      const int32_t inc = block_inclusive_scan<kGiantNT>(t, ws, &total);
      int32_t run = inc - t;
#pragma unroll
      for (int q = 0; q < P; ++q) {
        sub[threadIdx.x * P + q] = run;
        run += v[q];
      }
      __syncthreads();
    }
    cta_walk<kGiantNT, 4>(w, k0, k1, s_beg, s_pref, ws, [&](int32_t f) {
      wl[atomicAdd(sub + ((f - f_lo) >> shift), 1)] = f;
    });
    // now sub[b] = end of sub-range b = start of b + 1
    // 3. bucket starts: sub-range b opens a bucket when start(b) / cap changes
    {
      constexpr int P = kNSB / kGiantNT;
      int32_t flag[P], t = 0;
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int32_t b = threadIdx.x * P + q;
        flag[q] = 0;
        if (b < nsb) {
          const int32_t st = b ? sub[b - 1] : 0;
          const int32_t sp = b > 1 ? sub[b - 2] : 0;
          flag[q] = (b == 0) || (st / cap != sp / cap);
        }
        t += flag[q];
      }
      int32_t total;
      const int32_t inc = block_inclusive_scan<kGiantNT>(t, ws, &total);
      int32_t pos = inc - t;
#pragma unroll
      for (int q = 0; q < P; ++q)
        if (flag[q]) bstart[pos++] = threadIdx.x * P + q;
      if (threadIdx.x == 0) {
        bstart[total] = nsb;
        s_misc[1] = total;
      }
      __syncthreads();
    }
    const int32_t nb = s_misc[1];
    long long base = -1;
    if (a.mode == kDirect) base = a.row_ptr[e - a.row_begin];
    int32_t out = 0;  // pairs of the row so far
    for (int32_t c = 0; c < nb; ++c) {
      const int32_t b0 = bstart[c], b1 = bstart[c + 1];
      const int32_t lo = b0 ? sub[b0 - 1] : 0, hi = sub[b1 - 1];
      const int32_t width = (b1 - b0) << shift;
      const int lgT = table_lg(min(hi - lo, width), lg_max);
      const int32_t T = 1 << lgT;
      for (int32_t i = lo + (int32_t)threadIdx.x; i < hi; i += kGiantNT)
        table_insert(keys, cnts, lgT, wl[i], 1, smin, unweighted, meta);
      __syncthreads();
      const int32_t total = table_collect<kGiantNT, kGiantSPT>(keys, cnts, T, smin, emit, ws);
      if (emit && total > 0) {
        const unsigned long long *sb = reinterpret_cast<const unsigned long long *>(keys);
        for (int32_t i = threadIdx.x; i < total; i += kGiantNT) {
          const unsigned long long x = sb[i];
          const int32_t f = (int32_t)(x >> 32), n = (int32_t)(uint32_t)x;
          if (a.mode == kDirect) {
            put(a, base, out + i, e, f, n);
          } else {
            tj[out + i] = f;
            if (!unweighted) tw[out + i] = n;
          }
        }
      }
      out += total;
      table_reset<kGiantNT, kGiantSPT>(keys, cnts, T);
    }
    if (threadIdx.x == 0) *s_base = reserve(a, e, out, kBinGiant);
    __syncthreads();
    if (a.mode == kStage) {
      const long long b = *s_base;
      if (b >= 0)
        for (int32_t i = threadIdx.x; i < out; i += kGiantNT) {
          a.stage_j[b + i] = tj[i];
          if (!unweighted) a.stage_w[b + i] = tw[i];
        }
    }
  }
}

// --------------------------------------------------------------- launch --

namespace {

using CfgS = CtaCfg<256, 2 * kCtaSMaxWork>;
using CfgL = CtaCfg<1024, 2 * kCtaLMaxWork>;
#define K_CTA_S k_walk_cta<256, 2 * kCtaSMaxWork, kBinCtaS>
#define K_CTA_L k_walk_cta<1024, 2 * kCtaLMaxWork, kBinCtaL>

struct Occ {
  int sms = 0, warp_blocks = 0, s_blocks = 0, l_blocks = 0, g_blocks = 0;
  int dev = -1;
};

Occ &occ_for_device() {
  static Occ occ[64];
  int dev = 0;
  cudaGetDevice(&dev);
  Occ &o = occ[dev & 63];
  if (o.dev != dev) {
    cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(K_CTA_S, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CfgS::smem());
    cudaFuncSetAttribute(K_CTA_L, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CfgL::smem());
    cudaFuncSetAttribute(k_walk_giant, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)giant_smem());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.warp_blocks, k_walk_warp, kWarpNT, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.s_blocks, K_CTA_S, 256, CfgS::smem());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.l_blocks, K_CTA_L, 1024, CfgL::smem());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.g_blocks, k_walk_giant, kGiantNT,
                                                  giant_smem());
    if (o.g_blocks < 1) o.g_blocks = 1;
    o.dev = dev;
  }
  return o;
}

}  // namespace

int giant_ctas_for_device() {
  Occ &o = occ_for_device();
  return o.sms * o.g_blocks;
}

int giant_ctas() { return giant_ctas_for_device(); }

cudaError_t launch_walk(const WalkLaunch &L, cudaStream_t st, int32_t *launches,
                        cudaEvent_t *ev) {
  Occ &o = occ_for_device();
  const int32_t *lists = L.bin_rows;
  const int64_t stride = L.rows;
  int n = 0;
  if (ev) cudaEventRecord(ev[0], st);
  k_walk_warp<<<o.sms * (o.warp_blocks > 0 ? o.warp_blocks : 1), kWarpNT, 0, st>>>(
      L.w, lists + 0 * stride, L.a);
  ++n;
  if (ev) cudaEventRecord(ev[1], st);
  K_CTA_S<<<o.sms * (o.s_blocks > 0 ? o.s_blocks : 1), 256, CfgS::smem(), st>>>(
      L.w, lists + 1 * stride, L.row_work, L.a);
  ++n;
  if (ev) cudaEventRecord(ev[2], st);
  K_CTA_L<<<o.sms * (o.l_blocks > 0 ? o.l_blocks : 1), 1024, CfgL::smem(), st>>>(
      L.w, lists + 2 * stride, L.row_work, L.a);
  ++n;
  if (ev) cudaEventRecord(ev[3], st);
  if (L.giant_scratch) {
    k_walk_giant<<<o.sms * o.g_blocks, kGiantNT, giant_smem(), st>>>(
        L.w, lists + 3 * stride, L.a, L.giant_scratch, L.giant_stride, L.R);
    ++n;
  }
  if (ev) cudaEventRecord(ev[4], st);
  if (launches) *launches += n;
  return cudaGetLastError();
}

}  // namespace slg
