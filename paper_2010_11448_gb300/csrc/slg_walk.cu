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

// -------------------------------------------------------------- CTA bins --

template <int NT, int T>
struct CtaCfg {
  static constexpr int kNT = NT;
  static constexpr int kT = T;            // hash slots
  static constexpr int kSB = T / 2;       // sort buffer (>= max pairs of a row)
  static constexpr int kSPT = T / NT;     // slots per thread
  // [s_base 16 B][sbuf kSB x 8 B][keys T][cnts T][s_beg NT][s_pref NT+1][ws NT/32+1]
  static constexpr size_t smem() {
    return 16 + (size_t)kSB * 8 + (size_t)T * 8 + (size_t)(2 * NT + 1 + NT / 32 + 1) * 4;
  }
};

template <int NT, int T, int BIN>
__global__ __launch_bounds__(NT) void k_walk_cta(Walk w, const int32_t *__restrict__ rows,
                                                 EmitArgs a) {
  using Cfg = CtaCfg<NT, T>;
  Meta *meta = a.meta;
  if (meta->err) return;
  extern __shared__ __align__(16) unsigned char smem[];
  long long *s_base = reinterpret_cast<long long *>(smem);
  unsigned long long *sbuf = reinterpret_cast<unsigned long long *>(smem + 16);
  int32_t *keys = reinterpret_cast<int32_t *>(sbuf + Cfg::kSB);
  int32_t *cnts = keys + T;
  int32_t *s_beg = cnts + T;
  int32_t *s_pref = s_beg + NT;
  int32_t *ws = s_pref + NT + 1;

  for (int i = threadIdx.x; i < T; i += NT) {
    keys[i] = kEmpty;
    cnts[i] = 0;
  }
  __syncthreads();
  const long long nrows = (long long)meta->rows_bin[BIN];
  const int32_t smin = a.smin;
  const bool unweighted = a.unweighted != 0;
  for (long long r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int32_t e = rows[r];
    // 1. walk and count
    cta_walk<NT, 4>(w, w.r_off[e], w.r_off[e + 1], s_beg, s_pref, ws, [&](int32_t f) {
      uint32_t h = hash_slot(f, (uint32_t)T);
      for (int probe = 0; probe < T; ++probe) {
        const int32_t k = *(volatile int32_t *)(keys + h);
        if (k == f) {
          if (!unweighted || *(volatile int32_t *)(cnts + h) < smin) atomicAdd(cnts + h, 1);
          return;
        }
        if (k == kEmpty) {
          const int32_t prev = atomicCAS(keys + h, kEmpty, f);
          if (prev == kEmpty || prev == f) {
            atomicAdd(cnts + h, 1);
            return;
          }
        }
        h = (h + 1 == (uint32_t)T) ? 0u : h + 1;
      }
      raise_error(meta, SLG_ERR_INVALID, kWhereHash);  // unreachable by binning
    });
    // 2. pairs of this row: slots with count >= s (each thread owns kSPT slots)
    const int32_t h0 = threadIdx.x * Cfg::kSPT;
    int32_t c = 0;
#pragma unroll 4
    for (int i = 0; i < Cfg::kSPT; ++i) c += (keys[h0 + i] != kEmpty) & (cnts[h0 + i] >= smin);
    int32_t total;
    const int32_t inc = block_inclusive_scan<NT>(c, ws, &total);
    if (a.mode != kCount && total > 0) {
      int32_t pos = inc - c;
      for (int i = 0; i < Cfg::kSPT; ++i) {
        const int32_t k = keys[h0 + i], n = cnts[h0 + i];
        if (k != kEmpty && n >= smin)
          sbuf[pos++] = ((unsigned long long)(uint32_t)k << 32) | (uint32_t)n;
      }
      int32_t n2 = 1;
      while (n2 < total) n2 <<= 1;
      for (int32_t i = total + threadIdx.x; i < n2; i += NT) sbuf[i] = ~0ull;
      __syncthreads();
      for (int32_t k = 2; k <= n2; k <<= 1) {
        for (int32_t jj = k >> 1; jj > 0; jj >>= 1) {
          for (int32_t i = threadIdx.x; i < n2; i += NT) {
            const int32_t ixj = i ^ jj;
            if (ixj > i) {
              const unsigned long long x = sbuf[i], y = sbuf[ixj];
              const bool up = (i & k) == 0;
              if ((x > y) == up) {
                sbuf[i] = y;
                sbuf[ixj] = x;
              }
            }
          }
          __syncthreads();
        }
      }
    }
    if (threadIdx.x == 0) *s_base = reserve(a, e, total, BIN);
    __syncthreads();
    const long long base = *s_base;
    if (a.mode != kCount && base >= 0) {
      for (int32_t i = threadIdx.x; i < total; i += NT) {
        const unsigned long long x = sbuf[i];
        put(a, base, i, e, (int32_t)(x >> 32), (int32_t)(uint32_t)x);
      }
    }
    // 3. reset the owned slots for the next row
    for (int i = 0; i < Cfg::kSPT; ++i) {
      keys[h0 + i] = kEmpty;
      cnts[h0 + i] = 0;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------- giant bin --

constexpr int kGiantNT = 512;

// Shared layout: s_base (16 B) | summary[nsw] | s_beg[NT] | s_pref[NT+1] |
// ws[NT/32+1] | s_row.
// Each summary word covers 1024 consecutive ids (32 groups of 32 counters).
__global__ __launch_bounds__(kGiantNT) void k_walk_giant(Walk w, const int32_t *__restrict__ rows,
                                                         EmitArgs a, int32_t *__restrict__ scratch,
                                                         int32_t R_pad) {
  Meta *meta = a.meta;
  if (meta->err) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int32_t nsw = R_pad >> 10;
  long long *s_base = reinterpret_cast<long long *>(smem);
  uint32_t *summary = reinterpret_cast<uint32_t *>(smem + 16);
  int32_t *s_beg = reinterpret_cast<int32_t *>(summary + nsw);
  int32_t *s_pref = s_beg + kGiantNT;
  int32_t *ws = s_pref + kGiantNT + 1;
  int32_t *s_row = ws + kGiantNT / 32 + 1;
  int32_t *cnt = scratch + (size_t)blockIdx.x * R_pad;  // all zero between rows

  for (int i = threadIdx.x; i < nsw; i += kGiantNT) summary[i] = 0;
  const unsigned nrows = (unsigned)meta->rows_bin[kBinGiant];
  const int32_t smin = a.smin;
  const bool unweighted = a.unweighted != 0;
  const int32_t wpt = (nsw + kGiantNT - 1) / kGiantNT;  // summary words per thread
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned t = atomicAdd(&meta->giant_ticket, 1u);
      *s_row = t < nrows ? rows[t] : -1;
    }
    __syncthreads();
    const int32_t e = *s_row;
    if (e < 0) break;
    cta_walk<kGiantNT, 4>(w, w.r_off[e], w.r_off[e + 1], s_beg, s_pref, ws, [&](int32_t f) {
      if (unweighted && *(volatile int32_t *)(cnt + f) >= smin) return;
      if (atomicAdd(cnt + f, 1) == 0) atomicOr(summary + (f >> 10), 1u << ((f >> 5) & 31));
    });
    // count pairs in this thread's contiguous summary words
    const int32_t w0 = threadIdx.x * wpt;
    const int32_t w1 = min(nsw, w0 + wpt);
    int32_t c = 0;
    for (int32_t sw = w0; sw < w1; ++sw) {
      uint32_t bits = summary[sw];
      while (bits) {
        const int g = __ffs(bits) - 1;
        bits &= bits - 1;
        // Counters are updated by L2 atomics: read them at L2 (.cg), never
        // from a possibly stale L1 line.
        const int4 *p = reinterpret_cast<const int4 *>(cnt + ((sw << 10) | (g << 5)));
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int4 x = __ldcg(p + q);
          c += (x.x >= smin) + (x.y >= smin) + (x.z >= smin) + (x.w >= smin);
        }
      }
    }
    int32_t total;
    const int32_t inc = block_inclusive_scan<kGiantNT>(c, ws, &total);
    if (threadIdx.x == 0) *s_base = reserve(a, e, total, kBinGiant);
    __syncthreads();
    const long long base = *s_base;
    int32_t t = inc - c;
    for (int32_t sw = w0; sw < w1; ++sw) {
      uint32_t bits = summary[sw];
      while (bits) {
        const int g = __ffs(bits) - 1;
        bits &= bits - 1;
        const int32_t f0 = (sw << 10) | (g << 5);
        int4 *p = reinterpret_cast<int4 *>(cnt + f0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int4 x = __ldcg(p + q);
          if (a.mode != kCount && base >= 0) {
            if (x.x >= smin) put(a, base, t++, e, f0 + 4 * q + 0, x.x);
            if (x.y >= smin) put(a, base, t++, e, f0 + 4 * q + 1, x.y);
            if (x.z >= smin) put(a, base, t++, e, f0 + 4 * q + 2, x.z);
            if (x.w >= smin) put(a, base, t++, e, f0 + 4 * q + 3, x.w);
          }
          __stcg(p + q, make_int4(0, 0, 0, 0));
        }
      }
      summary[sw] = 0;
    }
  }
}

// --------------------------------------------------------------- launch --

namespace {

using CfgS = CtaCfg<256, 2 * kCtaSMaxWork>;
using CfgL = CtaCfg<1024, 2 * kCtaLMaxWork>;

struct Occ {
  int sms = 0, warp_blocks = 0, s_blocks = 0, l_blocks = 0, g_blocks = 0;
  int giant_smem_set = 0;
  int dev = -1;
};

Occ &occ_for_device() {
  static Occ occ[64];
  int dev = 0;
  cudaGetDevice(&dev);
  Occ &o = occ[dev & 63];
  if (o.dev != dev) {
    cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_walk_cta<256, 2 * kCtaSMaxWork, kBinCtaS>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CfgS::smem());
    cudaFuncSetAttribute(k_walk_cta<1024, 2 * kCtaLMaxWork, kBinCtaL>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CfgL::smem());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.warp_blocks, k_walk_warp, kWarpNT, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &o.s_blocks, k_walk_cta<256, 2 * kCtaSMaxWork, kBinCtaS>, 256, CfgS::smem());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &o.l_blocks, k_walk_cta<1024, 2 * kCtaLMaxWork, kBinCtaL>, 1024, CfgL::smem());
    o.g_blocks = 2;
    o.dev = dev;
  }
  return o;
}

}  // namespace

int giant_ctas_for_device() {
  Occ &o = occ_for_device();
  return o.sms * o.g_blocks;
}

size_t giant_smem_bytes(int32_t R_pad) {
  return 16 + (size_t)(R_pad >> 10) * 4 + (size_t)(2 * kGiantNT + 1 + kGiantNT / 32 + 1 + 1) * 4;
}

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
  k_walk_cta<256, 2 * kCtaSMaxWork, kBinCtaS><<<o.sms * (o.s_blocks > 0 ? o.s_blocks : 1), 256,
                                                CfgS::smem(), st>>>(L.w, lists + 1 * stride, L.a);
  ++n;
  if (ev) cudaEventRecord(ev[2], st);
  k_walk_cta<1024, 2 * kCtaLMaxWork, kBinCtaL><<<o.sms * (o.l_blocks > 0 ? o.l_blocks : 1), 1024,
                                                 CfgL::smem(), st>>>(L.w, lists + 2 * stride, L.a);
  ++n;
  if (ev) cudaEventRecord(ev[3], st);
  const size_t gsm = giant_smem_bytes(L.R_pad);
  if (gsm > (size_t)o.giant_smem_set) {
    cudaFuncSetAttribute(k_walk_giant, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
    o.giant_smem_set = (int)gsm;
  }
  k_walk_giant<<<L.giant_ctas, kGiantNT, gsm, st>>>(L.w, lists + 3 * stride, L.a,
                                                    L.giant_scratch, L.R_pad);
  ++n;
  if (ev) cudaEventRecord(ev[4], st);
  if (launches) *launches += n;
  return cudaGetLastError();
}

}  // namespace slg
