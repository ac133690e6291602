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
//   giant bin  (work > 8192):   a CTA splits the row's far ends into f-range
//                               buckets through a per-CTA global scratch and
//                               counts each bucket, in ascending f, in the
//                               shared-memory table.
//
// Output modes: COUNT (pairs per row only), STAGE (each row's sorted pairs
// are appended to a staging area at an atomically reserved offset) and
// DIRECT (written to their final place, row_ptr known).
#include <algorithm>
#include <mutex>
#include <type_traits>

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
    if (a.out_i) a.out_i[base + t] = e;  // null: compressed row form, i implied
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
    const int32_t smin = s_of(a.row_s, a.smin, e);
    // 1. gather the wedge ends (row work <= kWarpBuf by binning)
    int32_t filled = 0;
    for (int32_t base = k0; base < k1; base += 32) {
      const int32_t k = base + lane;
      int32_t b = 0, len = 0;
      if (k < k1) {
        b = __ldg(w.tail_beg + k);
        len = __ldg(w.tail_end + k) - b;
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
        q = (end - p) >= smin;
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
          q = c >= smin;
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
// An open-addressing table of T = 2^lgT 64-bit slots in shared memory, each
// slot (f << 32 | count) for a far end f; kEmpty64 marks a free slot.  The
// table holds at least twice the distinct keys it will receive, so it never
// fills.  A new key costs one CAS, a repeated one a 32-bit add to the slot's
// count word (see table_insert).  After the walk the slots with count >= s (found
// from the survivor list for s >= 2, by a pass over the table for s = 1) are
// moved to the front of the table, already packed as sort keys, and sorted
// by f.

constexpr unsigned long long kEmpty64 = 0xFFFFFFFF00000000ull;

// Survivor list (s >= 2): a key whose count reaches s during the inserts
// appends its slot to `slot` (one extra shared atomic per surviving pair),
// so collecting the survivors needs no pass over the table.  Counts only
// grow, so each key crosses s exactly once.  `cap` bounds the list (a
// survivor takes at least two wedges, or is one of at most T/2 keys).
struct SurvList {
  int32_t *slot;
  int32_t *n;
  int32_t cap;
};

__device__ __forceinline__ void note_survivor(const SurvList &sl, uint32_t h, int32_t old,
                                              int32_t add, int32_t smin, Meta *meta) {
  if (old < smin && old + add >= smin) {
    const int32_t p = atomicAdd(sl.n, 1);
    if (p < sl.cap) sl.slot[p] = (int32_t)h;
    else raise_error(meta, SLG_ERR_INVALID, kWhereHash);  // unreachable by the bound
  }
}

// The count word of slot h: its low 32 bits (the key word is the high half).
// Counts grow by 32-bit atomic adds, several times faster than 64-bit ones
// in shared memory on this GPU.
__device__ __forceinline__ uint32_t *count_word(unsigned long long *tab, uint32_t h) {
  return reinterpret_cast<uint32_t *>(tab + h);
}

// Inserts `add` wedges to far end f.  Unweighted: a count that reached s is
// not raised further.
//  - With the survivor list (s >= 2; mostly new keys in sparse rows) the key
//    word alone is claimed with a 32-bit CAS and the claim itself stands for
//    one wedge: the count word holds count - 1 (table_collect_list adds the
//    1 back).  A repeated key adds to the count word.
//  - Otherwise a probe reads the slot first (sparing repeated keys the CAS)
//    and a new key is claimed with one 64-bit CAS that also sets its count.
template <bool LIST>
__device__ __forceinline__ void table_insert(unsigned long long *tab, int lgT, int32_t f,
                                             int32_t add, int32_t smin, bool unweighted,
                                             Meta *meta, const SurvList &sl) {
  const uint32_t mask = (1u << lgT) - 1u;
  const unsigned long long key = (unsigned long long)(uint32_t)f << 32;
  uint32_t h = ((uint32_t)f * 0x9E3779B1u) >> (32 - lgT);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    if (LIST) {
      uint32_t *cw = count_word(tab, h);
      const uint32_t k = atomicCAS(cw + 1, 0xFFFFFFFFu, (uint32_t)f);  // key word
      if (k == 0xFFFFFFFFu) {  // claimed: count 1 so far
        if (add > 1) {
          const int32_t old = (int32_t)atomicAdd(cw, (uint32_t)(add - 1));
          note_survivor(sl, h, old + 1, add - 1, smin, meta);
        }
        return;
      }
      if (k == (uint32_t)f) {
        if (unweighted && (int32_t)*(volatile uint32_t *)cw + 1 >= smin) return;
        const int32_t old = (int32_t)atomicAdd(cw, (uint32_t)add);
        note_survivor(sl, h, old + 1, add, smin, meta);
        return;
      }
      h = (h + 1) & mask;
      continue;
    }
    unsigned long long cur = *(volatile unsigned long long *)(tab + h);
    if (cur == kEmpty64) {
      cur = atomicCAS(tab + h, kEmpty64, key | (uint32_t)add);
      if (cur == kEmpty64) return;
    }
    if ((cur & kEmpty64) == key) {
      if (!unweighted || (int32_t)(uint32_t)cur < smin) atomicAdd(count_word(tab, h), (uint32_t)add);
      return;
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

// Ascending order of one key per lane across a warp: a bitonic network on
// shuffles (for k = 32 every lane is in an ascending half).
__device__ __forceinline__ unsigned long long warp_sort32(unsigned long long x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, j);
      const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
      x = keep_min ? (x < y ? x : y) : (x < y ? y : x);
    }
  return x;
}

// Number of keys below x in a sorted run a[0, 32): branch-free binary search.
__device__ __forceinline__ int32_t run_below(const unsigned long long *a, unsigned long long x) {
  int32_t c = 0;
#pragma unroll
  for (int st = 16; st > 0; st >>= 1)
    if (a[c + st - 1] < x) c += st;
  return c + (a[c] < x);  // adds one only when c = 31 and all 32 are below
}

// Sorts the distinct keys tab[0, n) by f and returns where they are.
//  - small n (<= 64 with 512 threads, <= 512 with fewer): each key's rank is
//    the number of keys below it (one broadcast pass), written to [n, 2 n);
//  - 512 threads, n <= 1024: each warp sorts runs of 32 keys in registers
//    (padding ~0, above every key) and stores them back; a key's place is
//    then the sum over all runs of the keys below it (its own run contributes
//    its index), written to [32 nr, 32 nr + n) for nr = ceil(n / 32) runs.
//    (Smaller blocks keep the rank pass: the run code's registers would cost
//    them a resident block per SM.)
//  - larger n: a bitonic sort in place over [0, n2), n2 = 2^ceil(log2 n).
// `*used` receives the end of the region touched; it stays within
// max(T, 2 n + 32) <= the table's capacity for T >= 2 n.
template <int NT, bool RUNS = (NT >= 512)>
__device__ __forceinline__ int32_t sort_survivors(unsigned long long *tab, int32_t n,
                                                  int32_t *used) {
  constexpr bool kRuns = RUNS;
  if (n <= (kRuns ? 64 : 512)) {
    for (int32_t i = threadIdx.x; i < n; i += NT) {
      const unsigned long long x = tab[i];
      int32_t r = 0;
      for (int32_t j = 0; j < n; ++j) r += tab[j] < x;
      tab[n + r] = x;
    }
    __syncthreads();
    *used = 2 * n;
    return n;
  }
  if constexpr (kRuns) {
    if (n <= 8 * NT) {
      const int32_t nr = (n + 31) >> 5;
      for (int32_t r = (int32_t)threadIdx.x >> 5; r < nr; r += NT / 32) {
        const int32_t i = (r << 5) + (int32_t)(threadIdx.x & 31);
        const unsigned long long x = warp_sort32(i < n ? tab[i] : ~0ull);
        tab[i] = x;  // the run's loads precede the shuffles
      }
      __syncthreads();
      const int32_t out = nr << 5;
      for (int32_t i = threadIdx.x; i < n; i += NT) {
        const unsigned long long x = tab[i];
        int32_t r = 0;
        int32_t q = 0;
        for (; q + 4 <= nr; q += 4) {
          const int32_t c0 = run_below(tab + (q << 5), x);
          const int32_t c1 = run_below(tab + ((q + 1) << 5), x);
          const int32_t c2 = run_below(tab + ((q + 2) << 5), x);
          const int32_t c3 = run_below(tab + ((q + 3) << 5), x);
          r += c0 + c1 + c2 + c3;
        }
        for (; q < nr; ++q) r += run_below(tab + (q << 5), x);
        tab[out + r] = x;
      }
      __syncthreads();
      *used = out + n;
      return out;
    }
  }
  int32_t n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int32_t i = n + threadIdx.x; i < n2; i += NT) tab[i] = ~0ull;
  __syncthreads();
  for (int32_t k = 2; k <= n2; k <<= 1) {
    for (int32_t jj = k >> 1; jj > 0; jj >>= 1) {
      for (int32_t i = threadIdx.x; i < n2; i += NT) {
        const int32_t ixj = i ^ jj;
        if (ixj > i) {
          const unsigned long long x = tab[i], y = tab[ixj];
          if ((x > y) == ((i & k) == 0)) {
            tab[i] = y;
            tab[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  *used = n2;
  return 0;
}

// fn(r, x) for every key x of k[0, n) with r = the number of keys below x
// (distinct keys): for n <= 64 (or always, without RUNS) by one broadcast
// pass, else from runs of 32
// sorted in place (k[0, 32 ceil(n / 32)) is overwritten, padded with ~0)
// and binary searches over them.  No barrier after the calls.
template <int NT, bool RUNS = true, class Fn>
__device__ __forceinline__ void rank_keys(unsigned long long *k, int32_t n, Fn &&fn) {
  if (!RUNS || n <= 64) {
    for (int32_t i = threadIdx.x; i < n; i += NT) {
      const unsigned long long x = k[i];
      int32_t r = 0;
      for (int32_t j = 0; j < n; ++j) r += k[j] < x;
      fn(r, x);
    }
    return;
  }
  if constexpr (!RUNS) return;
  const int32_t nr = (n + 31) >> 5;
  for (int32_t q = (int32_t)threadIdx.x >> 5; q < nr; q += NT / 32) {
    const int32_t i = (q << 5) + (int32_t)(threadIdx.x & 31);
    const unsigned long long x = warp_sort32(i < n ? k[i] : ~0ull);
    k[i] = x;  // the run's loads precede the shuffles
  }
  __syncthreads();
  // runs 0 .. nr-2 are full and the last one holds its keys first, so
  // k[0, n) holds every key once
  for (int32_t i = threadIdx.x; i < n; i += NT) {
    const unsigned long long x = k[i];
    int32_t r = 0;
    for (int32_t q = 0; q < nr; ++q) r += run_below(k + (q << 5), x);
    fn(r, x);
  }
}

// Survivors by a pass over the table (used for s = 1, where every key
// survives).
// Rounds of RND slots per thread (slot = (round * RND + i) * NT + thread):
// a round reads its slots into registers, a block scan places the ones that
// qualify, and they are written to the front of the table.  A write of round
// r lands below the number of qualifying slots seen so far, hence on a slot
// of round r or earlier, all of which were read before the round's scan.
// Returns the number of survivors; with `sort` they are in ascending f at
// tab[*sorted_at, *sorted_at + count), and tab[0, *used) must be cleared
// after use (table_reset_front).
template <int NT, int SPT, bool RUNS = (NT >= 512)>
__device__ __forceinline__ int32_t table_collect(unsigned long long *tab, int32_t T, int32_t smin,
                                                 bool sort, int32_t *ws, int32_t *sorted_at,
                                                 int32_t *used, int32_t sort_cap = 0x7fffffff) {
  constexpr int RND = SPT < 8 ? SPT : 8;
  int32_t run = 0;
  for (int32_t r0 = 0; r0 * NT < T; r0 += RND) {
    unsigned long long kv[RND];
    int32_t c = 0;
#pragma unroll
    for (int i = 0; i < RND; ++i) {
      const int32_t slot = (r0 + i) * NT + (int32_t)threadIdx.x;
      kv[i] = slot < T ? tab[slot] : kEmpty64;
      c += (kv[i] != kEmpty64) & ((int32_t)(uint32_t)kv[i] >= smin);
    }
    int32_t total;
    const int32_t inc = block_inclusive_scan<NT>(c, ws, &total);  // the round's reads done
    if (sort) {
      int32_t pos = run + inc - c;
#pragma unroll
      for (int i = 0; i < RND; ++i)
        if (kv[i] != kEmpty64 && (int32_t)(uint32_t)kv[i] >= smin) tab[pos++] = kv[i];
    }
    run += total;
  }
  *used = T;
  if (sort && run > sort_cap) return -1;  // uniform: too many to order in the table
  if (sort && run > 0) {
    __syncthreads();  // compaction writes done
    int32_t u;
    *sorted_at = sort_survivors<NT, RUNS>(tab, run, &u);
    *used = max(T, u);
  }
  return run;
}

// Marks tab[0, n) free with 16-byte stores (tab is 16-byte aligned; an odd n
// also clears slot n, which is free already or inside the region in use).
template <int NT>
__device__ __forceinline__ void clear_slots(unsigned long long *tab, int32_t n) {
  ulonglong2 *t2 = reinterpret_cast<ulonglong2 *>(tab);
  const ulonglong2 e = make_ulonglong2(kEmpty64, kEmpty64);
  for (int32_t i = threadIdx.x; i < (n + 1) >> 1; i += NT) t2[i] = e;
}

// Survivors from the list: read their (f, count) slots, clear the whole
// table (plain stores), and with `sort` place them compactly at the front
// and sort them.  Returns the number of survivors; with `sort` they are in
// ascending f at tab[*sorted_at, + count) and tab[0, *used) must be cleared
// after use (table_reset_front).  QMAX x NT >= the list's capacity.
template <int NT, int QMAX>
__device__ __forceinline__ int32_t table_collect_list(unsigned long long *tab, int32_t T,
                                                      const SurvList &sl, bool sort,
                                                      int32_t *sorted_at, int32_t *used) {
  __syncthreads();  // every insert done: the list is final
  const int32_t n = min(*sl.n, sl.cap);
  unsigned long long x[QMAX];
#pragma unroll
  for (int q = 0; q < QMAX; ++q) {
    const int32_t i = (int32_t)threadIdx.x + q * NT;
    x[q] = (sort && i < n) ? tab[sl.slot[i]] + 1ull : 0ull;  // count word holds count - 1
  }
  __syncthreads();  // reads done before the table is cleared
  clear_slots<NT>(tab, T);
  if (threadIdx.x == 0) *sl.n = 0;
  __syncthreads();
  *used = 0;
  *sorted_at = 0;
  if (!sort || n == 0) return n;
#pragma unroll
  for (int q = 0; q < QMAX; ++q) {
    const int32_t i = (int32_t)threadIdx.x + q * NT;
    if (i < n) tab[i] = x[q];
  }
  __syncthreads();
  *sorted_at = sort_survivors<NT>(tab, n, used);
  return n;
}

// Clears tab[0, used) after the survivors were emitted.
template <int NT>
__device__ __forceinline__ void table_reset_front(unsigned long long *tab, int32_t used) {
  __syncthreads();  // sorted entries may still be read
  clear_slots<NT>(tab, used);
  __syncthreads();
}

// -------------------------------------------------------------- CTA bins --

#ifndef SLG_CTA_LIST_SORT
#define SLG_CTA_LIST_SORT 1
#endif
template <int NT, int TMAX>
struct CtaCfg {
  static constexpr int kSPT = TMAX / NT;  // slots per thread at most
  static constexpr int kList = TMAX / 4;  // survivors of a row when s >= 2 (<= work / 2)
  static constexpr int kQ = (kList + NT - 1) / NT;
  // survivor sets ranked in the list area: ceil(n / 2) + n keys <= kList / 2
  static constexpr int kListSortMax = kList / 3;
  static_assert((16 + TMAX * 8 + (2 * NT + 1 + NT / 32 + 1) * 4) % 8 == 0,
                "the survivor list starts on an 8-byte boundary");
  // [s_base 16 B][table TMAX x 8 B][s_beg NT][s_pref NT+1][ws NT/32+1]
  // [list kList][list count 1]
  static constexpr size_t smem() {
    return 16 + (size_t)TMAX * 8 + (size_t)(2 * NT + 1 + NT / 32 + 1) * 4 +
           (size_t)(kList + 1) * 4;
  }
};

template <int NT, int TMAX, int BIN, int MINB>
__global__ __launch_bounds__(NT, MINB) void k_walk_cta(Walk w, const int32_t *__restrict__ rows,
                                                 const int32_t *__restrict__ row_work,
                                                 EmitArgs a) {
  using Cfg = CtaCfg<NT, TMAX>;
  Meta *meta = a.meta;
  if (meta->err) return;
  extern __shared__ __align__(16) unsigned char smem[];
  long long *s_base = reinterpret_cast<long long *>(smem);
  unsigned long long *tab = reinterpret_cast<unsigned long long *>(smem + 16);
  int32_t *s_beg = reinterpret_cast<int32_t *>(tab + TMAX);
  int32_t *s_pref = s_beg + NT;
  int32_t *ws = s_pref + NT + 1;
  const SurvList sl = {ws + NT / 32 + 1, ws + NT / 32 + 1 + Cfg::kList, Cfg::kList};
  constexpr int lg_max = (TMAX >= 2) ? 31 - __builtin_clz(TMAX) : 1;

  for (int i = threadIdx.x; i < TMAX; i += NT) tab[i] = kEmpty64;
  if (threadIdx.x == 0) *sl.n = 0;
  __syncthreads();
  const long long nrows = (long long)meta->rows_bin[BIN];
  const bool unweighted = a.unweighted != 0;
  const bool emit = a.mode != kCount;
  for (long long r = blockIdx.x; r < nrows; r += gridDim.x) {
    const int32_t e = rows[r];
    const int32_t smin = s_of(a.row_s, a.smin, e);
    const int lgT = table_lg(row_work[e - a.row_begin], lg_max);
    const int32_t T = 1 << lgT;
    const int32_t k0 = w.r_off[e], k1 = w.r_off[e + 1];
    int32_t at = 0, used = 0, total;
    // s >= 2: survivors are listed as they appear; s = 1: every key survives
    if (smin >= 2) {
      cta_walk<NT, 4>(w, k0, k1, s_beg, s_pref, ws, [&](int32_t f, int32_t) {
        table_insert<true>(tab, lgT, f, 1, smin, unweighted, meta, sl);
      });
#if SLG_CTA_LIST_SORT
      // as in the giant bin: survivors ranked in the list area while the
      // table is cleared, each written straight to its place
      __syncthreads();  // inserts done: the list is final
      const int32_t nl = min(*sl.n, sl.cap);
      if (emit && nl <= Cfg::kListSortMax) {  // uniform
        if (threadIdx.x == 0) *s_base = reserve(a, e, nl, BIN);
        unsigned long long *lk = reinterpret_cast<unsigned long long *>(sl.slot) + ((nl + 1) >> 1);
        for (int32_t i = threadIdx.x; i < nl; i += NT) lk[i] = tab[sl.slot[i]] + 1ull;
        __syncthreads();  // keys and base in place; every table and slot read done
        clear_slots<NT>(tab, T);
        if (threadIdx.x == 0) *sl.n = 0;
        const long long base = *s_base;
        if (base >= 0)
          rank_keys<NT, false>(lk, nl, [&](int32_t r, unsigned long long x) {
            put(a, base, r, e, (int32_t)(x >> 32), (int32_t)(uint32_t)x);
          });
        __syncthreads();  // keys and base read before the next row
        continue;
      }
#endif
      total = table_collect_list<NT, Cfg::kQ>(tab, T, sl, emit, &at, &used);
    } else {
      cta_walk<NT, 4>(w, k0, k1, s_beg, s_pref, ws, [&](int32_t f, int32_t) {
        table_insert<false>(tab, lgT, f, 1, smin, unweighted, meta, sl);
      });
      total = table_collect<NT, Cfg::kSPT>(tab, T, smin, emit, ws, &at, &used);
    }
    if (threadIdx.x == 0) *s_base = reserve(a, e, total, BIN);
    __syncthreads();
    const long long base = *s_base;
    if (emit && base >= 0) {
      for (int32_t i = threadIdx.x; i < total; i += NT) {
        const unsigned long long x = tab[at + i];
        put(a, base, i, e, (int32_t)(x >> 32), (int32_t)(uint32_t)x);
      }
    }
    table_reset_front<NT>(tab, used);
  }
}

// ------------------------------------------------------------ sparse bin --
//
// Large rows whose far ends are sparse in their id span, with s >= 2.  Almost
// every far end of such a row occurs once (on the Chung-Lu workloads about
// 96 % of the wedges of these rows are the only wedge to their far end), and
// a far end with a single wedge can never reach s >= 2.  The row is counted
// in two passes with little shared memory, so that several rows are in
// flight on each SM (the walk's far-end gathers are latency-bound: a row at
// a time per SM leaves the memory system idle):
//   1. every wedge sets its far end's bit in a one-hash Bloom filter (one
//      shared atomicOr); a wedge that finds the bit already set makes f a
//      candidate: f is claimed in a small shared table (key, count 0) and
//      marked in a second filter.  Every f with two or more wedges becomes
//      a candidate (its second wedge finds the bit set); so may a few
//      single-wedge f whose bit another f had set;
//   2. a second pass counts, exactly, every wedge whose far end is a
//      candidate (the second filter screens out almost all others before
//      the table is probed).  The count of f is then |e ∩ f|.  It reads the
//      row's far ends from a copy the first walk wrote to global scratch
//      (or, for a row of at most kSpCache wedges, to shared memory), or
//      walks the tails again when there is no room for the copy.
// The candidates with count >= s are sorted and emitted.  A row whose
// candidates overflow the table (a probe sequence longer than kSpMaxProbe)
// is handed to the giant bin, which runs after this one.
// Two instances of the kernel share the bin: rows above kSparseBigWork go
// to one with a 2^SLG_SP_LGT-slot table, the rest to one with a
// 2^SLG_SP_SMALL_LGT-slot table, whose smaller shared memory leaves room for
// one more resident CTA per SM.  Rows of up to 8192 wedges seldom have more
// candidates or survivors than the smaller table holds (the overflow would
// send them to the giant bin); rows of up to 16384 do.

#ifndef SLG_SP_NT
#define SLG_SP_NT 256
#endif
#ifndef SLG_SP_LOGB
#define SLG_SP_LOGB 17
#endif
#ifndef SLG_SP_LGT
#define SLG_SP_LGT 12
#endif
#ifndef SLG_SP_CACHE
#define SLG_SP_CACHE 0
#endif
#ifndef SLG_SP_MINB
#define SLG_SP_MINB 4
#endif
#ifndef SLG_SP_SMALL_LGT
#define SLG_SP_SMALL_LGT 11
#endif
#ifndef SLG_SP_SMALL_MINB
#define SLG_SP_SMALL_MINB 5
#endif
#ifndef SLG_SP_G
#define SLG_SP_G 6
#endif
#ifndef SLG_SP_RUNS
#define SLG_SP_RUNS 1  // order survivor sets above 64 by sorted warp runs
#endif
constexpr int kSpNT = SLG_SP_NT;
constexpr int kSpLogB = SLG_SP_LOGB;          // Bloom filter bits (log2)
constexpr int kSpWords = 1 << (kSpLogB - 5);
constexpr int kSpCWords = kSpWords / 4;       // candidate filter words
constexpr int kSpLgT = SLG_SP_LGT;            // candidate table slots (log2)
constexpr int kSpSmallLgT = SLG_SP_SMALL_LGT;  // the same, rows up to kSparseBigWork
constexpr int kSpCache = SLG_SP_CACHE;        // far ends kept of a small row
constexpr int kSpMaxProbe = 32;
constexpr int kSpG = SLG_SP_G;                // wedges per thread per walk step
static_assert((1 << kSpSmallLgT) >= kSpNT && kSpSmallLgT <= kSpLgT &&
                  kSpWords % (4 * kSpNT) == 0 && kSpCWords % 4 == 0,
              "sparse bin geometry");

// [s_base 8][s_ovf 4][s_row 4][pad 16][filter kSpWords x 4]
// [candidate filter kSpCWords x 4][table 2^lgt x 8][cache kSpCache x 4]
// [s_beg NT][s_pref NT+1][ws NT/32+1]
constexpr size_t sparse_smem(int lgt) {
  return 32 + (size_t)kSpWords * 4 + (size_t)kSpCWords * 4 + ((size_t)8 << lgt) +
         (size_t)kSpCache * 4 + (size_t)(2 * kSpNT + 1 + kSpNT / 32 + 1) * 4;
}

// A row's filter has 2^lgb bits (its candidate filter 2^(lgb - 2)) and its
// table 2^lgt slots, sized by the row's work (see sp_sizes).
__device__ __forceinline__ uint32_t sp_h1(int32_t f, int lgb) {  // Bloom filter bit
  return ((uint32_t)f * 0x9E3779B1u) >> (32 - lgb);
}
__device__ __forceinline__ uint32_t sp_h2(int32_t f, int lgb) {  // candidate filter bit
  return ((uint32_t)f * 0x85EBCA6Bu) >> (34 - lgb);
}
__device__ __forceinline__ uint32_t sp_ht(int32_t f, int lgt) {  // candidate table slot
  return ((uint32_t)f * 0xC2B2AE35u) >> (32 - lgt);
}

// Per-row sizes: a filter of >= 32 bits per wedge (so that a single-wedge
// far end finds its bit set by another with probability below 1/64 on
// average) and a table of >= one slot per wedge (every candidate has two
// wedges or is such a collision), within the shared-memory maxima (a table
// of at most 2^max_lgt slots).
__device__ __forceinline__ void sp_sizes(int32_t work, int max_lgt, int *lgb, int *lgt) {
  const int lw = ceil_log2(work > 1 ? work : 2);
  *lgb = min(max(lw + 5, 12), kSpLogB);
  *lgt = min(max(lw, 7), max_lgt);
}

// Pass 1: f is a candidate (its filter bit was already set).  Claims f's
// table slot (32-bit CAS on the key word; the count word stays 0) unless it
// is there already, and marks it in the candidate filter.  A probe sequence
// longer than kSpMaxProbe marks the row as overflowed.
__device__ __forceinline__ void sp_candidate(unsigned long long *tab, uint32_t *cand, int32_t f,
                                             int32_t *s_ovf, int lgb, int lgt) {
  if (*(volatile int32_t *)s_ovf) return;
  const uint32_t mask = (1u << lgt) - 1u;
  uint32_t h = sp_ht(f, lgt);
  for (int probe = 0; probe < kSpMaxProbe; ++probe) {
    const uint32_t k = atomicCAS(count_word(tab, h) + 1, 0xFFFFFFFFu, (uint32_t)f);
    if (k == 0xFFFFFFFFu) {
      const uint32_t c = sp_h2(f, lgb);
      atomicOr(cand + (c >> 5), 1u << (c & 31));
      return;
    }
    if (k == (uint32_t)f) return;
    h = (h + 1) & mask;
  }
  *(volatile int32_t *)s_ovf = 1;
}

// Pass 2, for an f that passed the candidate filter: counted if it is in
// the table.  Unweighted: a count that reached s is not raised further.
__device__ __forceinline__ void sp_count_listed(unsigned long long *tab, int32_t f, int32_t smin,
                                                bool unweighted, int lgt) {
  const uint32_t mask = (1u << lgt) - 1u;
  uint32_t h = sp_ht(f, lgt);
  for (int probe = 0; probe < kSpMaxProbe; ++probe) {
    uint32_t *cw = count_word(tab, h);
    const uint32_t k = cw[1];
    if (k == (uint32_t)f) {
      if (!unweighted || (int32_t)*(volatile uint32_t *)cw < smin) atomicAdd(cw, 1u);
      return;
    }
    if (k == 0xFFFFFFFFu) return;
    h = (h + 1) & mask;
  }
}

// Pass 2: one wedge to f; counted when f is a candidate.
__device__ __forceinline__ void sp_count(unsigned long long *tab, const uint32_t *cand,
                                         int32_t f, int32_t smin, bool unweighted, int lgb,
                                         int lgt) {
  const uint32_t c = sp_h2(f, lgb);
  if (!(cand[c >> 5] & (1u << (c & 31)))) return;
  sp_count_listed(tab, f, smin, unweighted, lgt);
}

// A lane's few wedges of a walk step that take the slow path (candidate
// claims in pass 1, counts in pass 2: a small fraction of the wedges) are
// gathered in registers and handled in rounds, the q-th round taking every
// lane's q-th one, so that a warp runs max over its lanes rounds instead of
// one round per wedge slot of the step with a lane or two active.
#ifndef SLG_SP_DEFER
#define SLG_SP_DEFER 1
#endif
template <int G>
__device__ __forceinline__ void pend_push(int32_t (&pend)[G], int &np, bool c, int32_t f, int g) {
#pragma unroll
  for (int q = 0; q < G; ++q)  // selects: no local memory
    if (q <= g) pend[q] = (c && q == np) ? f : pend[q];
  np += c;
}

// ------------------------------------------------------------- giant bin --
//
// A CTA takes one giant row at a time (dynamic ticket; rows above
// kGiantHugeWork wedges first, so that the schedule ends on small rows); two
// CTAs share an SM.  The row's far ends f lie in [f_lo, R) (f_lo = e + 1 for
// the upper-triangle walk, 0 for whole columns).  Rows of at most
// kGiantDirectMax wedges are counted in one table during the walk; the
// others are partitioned:
//   1. one load-balanced walk copies the row's far ends, in flattened wedge
//      order, to the CTA's global scratch `flat` (coalesced stores); a row
//      whose ids fit one super-chunk also counts its sub-range histogram
//      during this walk;
//   2. the id range is cut into super-chunks of at most kNSB sub-ranges of
//      2^shift ids each (2^shift <= kGiantTMax / 4).  Per super-chunk: a pass
//      over `flat` counts its wedges per sub-range (shared histogram), an
//      exclusive scan, and a second pass scatters them to `wl`, grouped by
//      sub-range;
//   3. consecutive sub-ranges form buckets of at most CAP wedges (a single
//      larger sub-range forms its own bucket: it holds at most 2^shift
//      distinct ids); bucket by bucket, in ascending f, the shared table
//      counts the far ends and the bucket's pairs (already in order) are
//      appended to the row's output.
// Core rows (tensor-core tile path) add their tile items (f, tile count) to
// the buckets of their id ranges.  Nothing is counted in global memory and
// the output comes out sorted.

// Geometry (compile-time; the defaults are the tuned values).
#ifndef SLG_GIANT_NT
#define SLG_GIANT_NT 512
#endif
#ifndef SLG_GIANT_TMAX
#define SLG_GIANT_TMAX 8192
#endif
#ifndef SLG_GIANT_MINB
#define SLG_GIANT_MINB 2
#endif
constexpr int kGiantNT = SLG_GIANT_NT;
constexpr int kGiantTMax = SLG_GIANT_TMAX;
constexpr int kNSBLog = 11;
constexpr int kNSB = 1 << kNSBLog;  // sub-ranges per super-chunk
constexpr int kShiftMax = 31 - __builtin_clz(kGiantTMax / 4);  // 2^shift <= kGiantTMax / 4
constexpr int kGiantSPT = kGiantTMax / kGiantNT;
constexpr int kDenseW = 2 * kGiantTMax;  // ids per dense window (int32 counters in the table)
// ids per dense window with 16-bit counters (rows of at most 65,535 vertices:
// a count |e ∩ f| never exceeds |e|)
constexpr int kDenseW16 = 4 * kGiantTMax;
#ifndef SLG_DENSE16
#define SLG_DENSE16 1
#endif

constexpr int kGiantList = kGiantTMax / 2;  // survivors of a bucket (<= its distinct keys)
#ifndef SLG_GIANT_DIRECT_MAX
#define SLG_GIANT_DIRECT_MAX 6144
#endif
// Rows of at most this many wedges skip the partition: one table, filled to
// at most 3/4 (the survivor list holds work / 2 >= any s >= 2 survivor set).
constexpr int32_t kGiantDirectMax = SLG_GIANT_DIRECT_MAX;
constexpr int kGiantG = 6;  // wedges per thread per step of the giant bin's walk (4, 6, 8 swept)
static_assert(kGiantDirectMax <= kGiantTMax && kGiantDirectMax / 2 <= kGiantList,
              "a direct row fits the table and the survivor list");
constexpr int kGiantQ = kGiantList / kGiantNT;
static_assert(kNSB % kGiantNT == 0 && kGiantTMax % kGiantNT == 0 && kGiantList % kGiantNT == 0,
              "giant bin geometry: whole sub-ranges, slots and list entries per thread");
// Survivor sets of up to this many keys are ordered in the survivor-list
// area (kGiantList ints = kGiantList / 2 keys): the keys start past the
// slot indices (ceil(n / 2) keys) and their runs take 32 ceil(n / 32).
#ifndef SLG_GIANT_LIST_SORT
#define SLG_GIANT_LIST_SORT 1
#endif
constexpr int32_t kGiantListSortMax = kGiantList / 4;
static_assert((kGiantListSortMax + 1) / 2 + 32 * ((kGiantListSortMax + 31) / 32) <=
                  kGiantList / 2,
              "the list area holds the runs of kGiantListSortMax keys");
static_assert(kGiantListSortMax <= 8 * kGiantNT, "the run sort covers the list sort");

// [s_base 16][s_misc 16][table TMAX x 8][sub NSB][subt NSB+1][bstart NSB+1]
// [s_beg NT][s_pref NT+1][ws NT/32+1][list kGiantList][list count 1]
constexpr size_t giant_smem() {
  return 32 + (size_t)kGiantTMax * 8 + (size_t)(3 * kNSB + 2) * 4 +
         (size_t)(2 * kGiantNT + 1 + kGiantNT / 32 + 1) * 4 + (size_t)(kGiantList + 1) * 4;
}
// The survivor list starts on an 8-byte boundary (it also holds 64-bit keys).
static_assert((32 + (size_t)kGiantTMax * 8 + (size_t)(3 * kNSB + 2) * 4 +
               (size_t)(2 * kGiantNT + 1 + kGiantNT / 32 + 1) * 4) % 8 == 0,
              "survivor list alignment");

// Drops from L2, without writing them back to DRAM, the 128-byte lines that
// lie wholly inside [p, p + n) (PTX discard.global.L2): for per-CTA scratch
// whose contents are dead.  Every reader of the range must have passed a
// block barrier since its last read; lines that the range shares with
// neighbouring data at its two ends are left alone.
__device__ __forceinline__ void l2_discard(const int32_t *p, long long n) {
  if (n <= 0) return;
  const unsigned long long g = (unsigned long long)__cvta_generic_to_global(p);
  const unsigned long long b = (g + 127ull) & ~127ull;
  const unsigned long long e = (g + 4ull * (unsigned long long)n) & ~127ull;
  for (unsigned long long x = b + 128ull * threadIdx.x; x < e; x += 128ull * blockDim.x)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(x) : "memory");
}

// Exclusive scan of the kNSB sub-range counters in place (P per thread);
// returns the total.
__device__ __forceinline__ int32_t scan_subranges(int32_t *a, int32_t *ws) {
  constexpr int P = kNSB / kGiantNT;
  int32_t v[P], t = 0;
#pragma unroll
  for (int q = 0; q < P; ++q) {
    v[q] = a[threadIdx.x * P + q];
    t += v[q];
  }
  int32_t total;
  const int32_t inc = block_inclusive_scan<kGiantNT>(t, ws, &total);
  int32_t run = inc - t;
#pragma unroll
  for (int q = 0; q < P; ++q) {
    a[threadIdx.x * P + q] = run;
    run += v[q];
  }
  __syncthreads();
  return total;
}

// fn(a[i]) for i = lo + threadIdx.x, lo + threadIdx.x + NT, ... < hi, with Q
// loads issued together before their first use (the scratch reads are
// latency-bound).
template <int NT, int Q, class Fn>
__device__ __forceinline__ void for_each_batched(const int32_t *a, int32_t lo, int32_t hi,
                                                 Fn &&fn) {
  for (int32_t i0 = lo + (int32_t)threadIdx.x; i0 < hi; i0 += Q * NT) {
    int32_t v[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int32_t i = i0 + q * NT;
      v[q] = i < hi ? a[i] : 0;
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
      if (i0 + q * NT < hi) fn(v[q]);
  }
}

// First position p in core_list[0, n) with core_list[p] >= x.
__device__ __forceinline__ int32_t core_lower(const int32_t *core_list, int32_t n, int32_t x) {
  int32_t a = 0, b = n;
  while (a < b) {
    const int32_t mid = (a + b) >> 1;
    if (__ldg(core_list + mid) < x) a = mid + 1;
    else b = mid;
  }
  return a;
}

__global__ __launch_bounds__(kGiantNT, SLG_GIANT_MINB) void k_walk_giant(Walk w, const int32_t *__restrict__ rows,
                                                            EmitArgs a, int32_t *__restrict__ scratch,
                                                            long long scratch_stride, int32_t R,
                                                            int32_t list_len) {
  Meta *meta = a.meta;
  if (meta->err) return;
  extern __shared__ __align__(16) unsigned char smem[];
  long long *s_base = reinterpret_cast<long long *>(smem);
  int32_t *s_misc = reinterpret_cast<int32_t *>(smem + 16);  // [0] row, [1] buckets, [2,3] items
  unsigned long long *tab = reinterpret_cast<unsigned long long *>(smem + 32);
  int32_t *sub = reinterpret_cast<int32_t *>(tab + kGiantTMax);
  int32_t *subt = sub + kNSB;  // tile items per sub-range (core rows)
  int32_t *bstart = subt + kNSB + 1;
  int32_t *s_beg = bstart + kNSB + 1;
  int32_t *s_pref = s_beg + kGiantNT;
  int32_t *ws = s_pref + kGiantNT + 1;
  const SurvList sl = {ws + kGiantNT / 32 + 1, ws + kGiantNT / 32 + 1 + kGiantList, kGiantList};
  // per-CTA global scratch, 4 ints per wedge of the largest row:
  // flattened far ends, far ends grouped by sub-range, staged pairs (j, w)
  const long long q4 = scratch_stride / 4;
  int32_t *flat = scratch + (long long)blockIdx.x * scratch_stride;
  int32_t *wl = flat + q4;
  int32_t *tj = wl + q4;
  int32_t *tw = tj + q4;

  for (int i = threadIdx.x; i < kGiantTMax; i += kGiantNT) tab[i] = kEmpty64;
  if (threadIdx.x == 0) *sl.n = 0;
  const unsigned nrows = (unsigned)meta->rows_bin[kBinGiant];
  const unsigned nhuge = meta->giant_huge;  // rows[0, nhuge); the others end at rows[list_len)
  const bool unweighted = a.unweighted != 0;
  const bool emit = a.mode != kCount;
  constexpr int lg_max = 31 - __builtin_clz(kGiantTMax);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned t = atomicAdd(&meta->giant_ticket, 1u);
      s_misc[0] = t >= nrows ? -1 : rows[t < nhuge ? t : list_len - 1 - (t - nhuge)];
    }
    __syncthreads();
    const int32_t e = s_misc[0];
    if (e < 0) break;
    const long long row_t0 = clock64();
    const int32_t smin = s_of(a.row_s, a.smin, e);
    const int32_t f_lo = a.full_rows ? 0 : e + 1;
    // far ends lie in [f_lo, f_hi): below R, or below the end of e's member
    // in a batched union
    const int32_t f_hi = a.row_fhi ? a.row_fhi[e] : R;
    const int32_t span = f_hi - f_lo;
    const int shift = min(kShiftMax, max(0, ceil_log2(span) - kNSBLog));
    const int32_t chunk_w = kNSB << shift;  // ids per super-chunk
    const int32_t cap = kGiantTMax / 2 - (1 << shift);
    const int32_t work = a.row_work[e - a.row_begin];
    // Dense rows (at least one wedge per 8 ids) count fixed windows of
    // kDenseW ids in a dense shared array: no hashing, no sort.
    const bool dense = (long long)work * a.dense_ratio >= (long long)span;
    // dense rows with 16-bit counters: twice the ids per window
    const bool d16 = SLG_DENSE16 && dense && w.r_off[e + 1] - w.r_off[e] <= 0xFFFF;
    const int32_t dwin = d16 ? kDenseW16 : kDenseW;
    if (work > q4) {  // the scratch is sized by the largest row: cannot happen
      if (threadIdx.x == 0) raise_error(meta, SLG_ERR_INVALID, kWhereGiant);
      break;
    }
    // Core rows also receive tile items (f, |e ∩ f ∩ C_c|) for every active
    // core row f > e with a non-zero tile count.
    const CoreInfo &ci = a.core;
    const bool core_row = ci.T && ci.row_rank[e + 1] != ci.row_rank[e];
    const int32_t ri = core_row ? ci.row_rank[e] : 0;
    const int32_t *Trow = core_row ? ci.T + (long long)ri * ci.Mp : nullptr;
    long long base = -1;
    if (a.mode == kDirect) base = a.row_ptr[e - a.row_begin];
    int32_t out = 0;  // pairs of the row so far
    if (work <= kGiantDirectMax && !core_row) {
      // A row this small is counted in one table during the walk, as in the
      // CTA bins (no flattened copy, no sub-ranges): its distinct far ends
      // fill at most kGiantDirectMax / kGiantTMax of the table.
      const int lgT = table_lg(work, lg_max);
      const int32_t T = 1 << lgT;
      int32_t at = 0, used = T;
      if (smin >= 2) {
        cta_walk<kGiantNT, kGiantG>(w, w.r_off[e], w.r_off[e + 1], s_beg, s_pref, ws,
                              [&](int32_t f, int32_t) {
                                table_insert<true>(tab, lgT, f, 1, smin, unweighted, meta, sl);
                              });
        out = table_collect_list<kGiantNT, kGiantQ>(tab, T, sl, emit, &at, &used);
      } else {
        cta_walk<kGiantNT, kGiantG>(w, w.r_off[e], w.r_off[e + 1], s_beg, s_pref, ws,
                              [&](int32_t f, int32_t) {
                                table_insert<false>(tab, lgT, f, 1, smin, unweighted, meta, sl);
                              });
        out = table_collect<kGiantNT, kGiantSPT>(tab, T, smin, emit, ws, &at, &used);
      }
      if (emit)
        for (int32_t i = threadIdx.x; i < out; i += kGiantNT) {
          const unsigned long long x = tab[at + i];
          const int32_t f = (int32_t)(x >> 32), n = (int32_t)(uint32_t)x;
          if (a.mode == kDirect) {
            put(a, base, i, e, f, n);
          } else {
            tj[i] = f;
            if (!unweighted) tw[i] = n;
          }
        }
      table_reset_front<kGiantNT>(tab, used);
    } else {
      long long clk0 = clock64();
      // 1. flattened far ends; a row within one super-chunk also counts its
      // sub-range histogram here (saving one pass over the copy)
      const bool single = f_hi - f_lo <= chunk_w;
      if (single) {
        for (int i = threadIdx.x; i < kNSB; i += kGiantNT) {
          sub[i] = 0;
          subt[i] = 0;
        }
        __syncthreads();
        cta_walk<kGiantNT, kGiantG>(w, w.r_off[e], w.r_off[e + 1], s_beg, s_pref, ws,
                              [&](int32_t f, int32_t i) {
                                flat[i] = f;
                                atomicAdd(sub + ((f - f_lo) >> shift), 1);
                              });
      } else {
        cta_walk<kGiantNT, kGiantG>(w, w.r_off[e], w.r_off[e + 1], s_beg, s_pref, ws,
                              [&](int32_t f, int32_t i) { flat[i] = f; });
      }
      long long clk_part = 0, clk_bucket = 0;
      if (threadIdx.x == 0) atomicAdd(&meta->giant_cycles[0], (unsigned long long)(clock64() - clk0));
      for (int32_t F0 = f_lo; F0 < f_hi; F0 += chunk_w) {
        // An empty bucket is skipped without a barrier, so threads may still
        // be reading the previous super-chunk's sub[] / bstart[] here: every
        // thread must be done with them before they are rewritten.
        __syncthreads();
        const long long c0 = clock64();
        const int32_t F1 = (f_hi - F0 > chunk_w) ? F0 + chunk_w : f_hi;
        const int32_t nsb = ((F1 - F0 - 1) >> shift) + 1;
        // 2. histograms of sub-ranges (wedges; tile items), scans, scatter
        if (!single) {
          for (int i = threadIdx.x; i < kNSB; i += kGiantNT) {
            sub[i] = 0;
            subt[i] = 0;
          }
          __syncthreads();
          for_each_batched<kGiantNT, 8>(flat, 0, work, [&](int32_t f) {
            if (f >= F0 && f < F1) atomicAdd(sub + ((f - F0) >> shift), 1);
          });
        }
        if (core_row)
          for (int32_t p = ri + 1 + (int32_t)threadIdx.x; p < ci.n_core; p += kGiantNT) {
            const int32_t f = ci.core_list[p];
            if (f >= F0 && f < F1 && w.r_off[f + 1] - w.r_off[f] >= smin && Trow[p] > 0)
              atomicAdd(subt + ((f - F0) >> shift), 1);
          }
        __syncthreads();
        const int32_t nw = scan_subranges(sub, ws);
        const int32_t items = core_row ? scan_subranges(subt, ws) : 0;
        if (nw == 0 && items == 0) continue;  // uniform: both totals are block-wide
        if (threadIdx.x == 0) subt[kNSB] = items;
        for_each_batched<kGiantNT, 8>(flat, 0, work, [&](int32_t f) {
          if (f >= F0 && f < F1) wl[atomicAdd(sub + ((f - F0) >> shift), 1)] = f;
        });
        __syncthreads();
        if (F1 == f_hi) l2_discard(flat, work);  // the flattened copy's last read
        // now sub[b] = end of the wedges of sub-range b; subt[b] = start of its
        // items.  3. bucket starts: sub-range b opens a bucket when its start
        // in the merged order (wedges + items before it) / cap changes.
        {
          constexpr int P = kNSB / kGiantNT;
          int32_t flag[P], t = 0;
  #pragma unroll
          for (int q = 0; q < P; ++q) {
            const int32_t b = threadIdx.x * P + q;
            flag[q] = 0;
            if (b < nsb) {
              if (dense) {
                flag[q] = ((b << shift) & (dwin - 1)) == 0;
              } else {
                const int32_t st = (b ? sub[b - 1] : 0) + (core_row ? subt[b] : 0);
                const int32_t sp = b ? (b > 1 ? sub[b - 2] : 0) + (core_row ? subt[b - 1] : 0) : 0;
                flag[q] = (b == 0) || (st / cap != sp / cap);
              }
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
        const long long c1 = clock64();
        clk_part += c1 - c0;
        for (int32_t c = 0; c < nb; ++c) {
          const int32_t b0 = bstart[c], b1 = bstart[c + 1];
          const int32_t lo = b0 ? sub[b0 - 1] : 0, hi = sub[b1 - 1];
          int32_t nit = 0;
          if (core_row) {
            nit = (b1 < nsb ? subt[b1] : subt[kNSB]) - subt[b0];
            if (threadIdx.x == 0) {
              // core positions of the bucket's id range, after row e itself
              const int32_t flo = F0 + (b0 << shift);
              const int32_t fhi = b1 < nsb ? F0 + (b1 << shift) : F1;
              s_misc[2] = max(core_lower(ci.core_list, ci.n_core, flo), ri + 1);
              s_misc[3] = core_lower(ci.core_list, ci.n_core, fhi);
            }
            __syncthreads();
          }
          if (hi - lo + nit == 0) continue;  // uniform
          if (d16) {
            // 16-bit counters, two per word; the emission scans 8 counters
            // per 16-byte load and reads a counter again only for survivors
            const int32_t fb0 = F0 + (b0 << shift);
            const int32_t dw = min((b1 - b0) << shift, F1 - fb0);  // <= kDenseW16
            uint32_t *c32 = reinterpret_cast<uint32_t *>(tab);
            const uint16_t *c16 = reinterpret_cast<const uint16_t *>(tab);
            uint4 *c128 = reinterpret_cast<uint4 *>(tab);
            for (int32_t i = threadIdx.x; i < (dw + 7) / 8; i += kGiantNT)
              c128[i] = make_uint4(0, 0, 0, 0);
            __syncthreads();
            for_each_batched<kGiantNT, 8>(wl, lo, hi, [&](int32_t f) {
              const int32_t o = f - fb0;
              atomicAdd(c32 + (o >> 1), 1u << ((o & 1) << 4));
            });
            if (core_row && nit > 0)
              for (int32_t p = s_misc[2] + (int32_t)threadIdx.x; p < s_misc[3]; p += kGiantNT) {
                const int32_t f = ci.core_list[p];
                const int32_t wt = Trow[p];
                if (wt > 0 && w.r_off[f + 1] - w.r_off[f] >= smin) {
                  const int32_t o = f - fb0;
                  atomicAdd(c32 + (o >> 1), (uint32_t)wt << ((o & 1) << 4));
                }
              }
            __syncthreads();
            // warp q owns counters [q * span_w, (q + 1) * span_w); lane l
            // takes the groups of 8 at q0 + 8 (l + 32 k), k < span_w / 256
            const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
            constexpr int NWq = kGiantNT / 32;
            constexpr int KMAX = kDenseW16 / NWq / 256;  // groups per lane at most
            const int32_t span_w = ((dw + NWq - 1) / NWq + 255) & ~255;
            const int32_t q0 = wq * span_w, q1 = min(dw, q0 + span_w);
            const int32_t nk = span_w >> 8;
            const uint32_t s2 = (uint32_t)min(smin, 0xFFFF) * 0x10001u;
            uint32_t mk[KMAX];
            int32_t c = 0;
  #pragma unroll
            for (int k = 0; k < KMAX; ++k) {
              mk[k] = 0;
              const int32_t i8 = q0 + ((lane + (k << 5)) << 3);
              if (k < nk && i8 < q1) {
                const uint4 v = c128[i8 >> 3];
                // per 16-bit counter: 0xFFFF where count >= smin
                const uint32_t g0 = __vcmpgeu2(v.x, s2), g1 = __vcmpgeu2(v.y, s2);
                const uint32_t g2 = __vcmpgeu2(v.z, s2), g3 = __vcmpgeu2(v.w, s2);
                mk[k] = (g0 & 1u) | ((g0 >> 15) & 2u) | ((g1 & 1u) << 2) | ((g1 >> 13) & 8u) |
                        ((g2 & 1u) << 4) | ((g2 >> 11) & 32u) | ((g3 & 1u) << 6) |
                        ((g3 >> 9) & 128u);
                c += __popc(mk[k]);
              }
            }
  #pragma unroll
            for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
            int32_t total;
            const int32_t winc = block_inclusive_scan<kGiantNT>(lane == 0 ? c : 0, ws, &total);
            int32_t pos = out + __shfl_sync(0xffffffffu, winc, 0) - c;  // warp's first slot
            if (a.mode == kStage && out + total > q4) {
              if (threadIdx.x == 0) raise_error(meta, SLG_ERR_INVALID, kWhereGiant);
              break;
            }
            if (emit && total > 0) {
  #pragma unroll
              for (int k = 0; k < KMAX; ++k) {
                if (k >= nk) break;  // warp-uniform
                uint32_t m = mk[k];
                const int32_t cnt = __popc(m);
                const int32_t inc = warp_inclusive_scan(cnt);
                int32_t t = pos + inc - cnt;
                pos += __shfl_sync(0xffffffffu, inc, 31);
                const int32_t i8 = q0 + ((lane + (k << 5)) << 3);
                while (m) {
                  const int b = __ffs(m) - 1;
                  m &= m - 1;
                  const int32_t i = i8 + b;
                  const int32_t n = c16[i];
                  if (a.mode == kDirect) {
                    put(a, base, t, e, fb0 + i, n);
                  } else {
                    tj[t] = fb0 + i;
                    if (!unweighted) tw[t] = n;
                  }
                  ++t;
                }
              }
            }
            out += total;
            __syncthreads();
            for (int32_t i = threadIdx.x; i < (dw + 3) / 4; i += kGiantNT) tab[i] = kEmpty64;
            __syncthreads();
            continue;
          }
          if (dense) {
            const int32_t fb0 = F0 + (b0 << shift);
            const int32_t dw = min((b1 - b0) << shift, F1 - fb0);  // <= kDenseW
            int32_t *cnt = reinterpret_cast<int32_t *>(tab);
            for (int32_t i = threadIdx.x; i < dw; i += kGiantNT) cnt[i] = 0;
            __syncthreads();
            for_each_batched<kGiantNT, 8>(wl, lo, hi,
                                          [&](int32_t f) { atomicAdd(cnt + (f - fb0), 1); });
            if (core_row && nit > 0)
              for (int32_t p = s_misc[2] + (int32_t)threadIdx.x; p < s_misc[3]; p += kGiantNT) {
                const int32_t f = ci.core_list[p];
                const int32_t wt = Trow[p];
                if (wt > 0 && w.r_off[f + 1] - w.r_off[f] >= smin) atomicAdd(cnt + (f - fb0), wt);
              }
            __syncthreads();
            // ordered emission: warp q owns counters [q * span_w, (q + 1) * span_w)
            const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
            constexpr int NWq = kGiantNT / 32;
            const int32_t span_w = ((dw + NWq - 1) / NWq + 31) & ~31;
            const int32_t q0 = wq * span_w, q1 = min(dw, q0 + span_w);
            int32_t c = 0;
            for (int32_t i = q0 + lane; i < q1; i += 32) c += cnt[i] >= smin;
  #pragma unroll
            for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
            int32_t total;
            const int32_t winc = block_inclusive_scan<kGiantNT>(lane == 0 ? c : 0, ws, &total);
            int32_t pos = out + __shfl_sync(0xffffffffu, winc, 0) - c;  // warp's first slot
            if (a.mode == kStage && out + total > q4) {
              if (threadIdx.x == 0) raise_error(meta, SLG_ERR_INVALID, kWhereGiant);
              break;
            }
            if (emit && total > 0) {
              for (int32_t i0 = q0; i0 < q1; i0 += 32) {
                const int32_t i = i0 + lane;
                const int32_t n = i < q1 ? cnt[i] : 0;
                const bool keep = i < q1 && n >= smin;
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                  const int32_t t = pos + __popc(bal & ((1u << lane) - 1));
                  if (a.mode == kDirect) {
                    put(a, base, t, e, fb0 + i, n);
                  } else {
                    tj[t] = fb0 + i;
                    if (!unweighted) tw[t] = n;
                  }
                }
                pos += __popc(bal);
              }
            }
            out += total;
            __syncthreads();
            for (int32_t i = threadIdx.x; i < (dw + 1) / 2; i += kGiantNT) tab[i] = kEmpty64;
            __syncthreads();
            continue;
          }
          // the sorted pairs tab[at, at + total) of a bucket go to the row's
          // output; false (uniform) when they would not fit the scratch
          auto emit_sorted = [&](int32_t at, int32_t total, int32_t used) -> bool {
            if (a.mode == kStage && out + total > q4) {
              // staged pairs would not fit the scratch (sized by wedges +
              // core items): report instead of writing past it
              if (threadIdx.x == 0) raise_error(meta, SLG_ERR_INVALID, kWhereGiant);
              table_reset_front<kGiantNT>(tab, used);
              return false;
            }
            if (emit && total > 0) {
              for (int32_t i = threadIdx.x; i < total; i += kGiantNT) {
                const unsigned long long x = tab[at + i];
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
            table_reset_front<kGiantNT>(tab, used);
            return true;
          };
          // sub-ranges [h0, h1) (wedges wl[hlo, hhi), tile items `hnit`)
          // counted in the hash table
          auto hash_bucket = [&](int32_t h0, int32_t h1, int32_t hlo, int32_t hhi,
                                 int32_t hnit) -> bool {
            const int32_t width = (h1 - h0) << shift;
            const int lgT = table_lg(min(hhi - hlo + hnit, width), lg_max);
            const int32_t T = 1 << lgT;
            // s >= 2: survivors listed as they appear; s = 1: every key survives
            const bool list = smin >= 2;
            auto insert_all = [&](auto list_tag) {
              constexpr bool L = decltype(list_tag)::value;
              for_each_batched<kGiantNT, 8>(wl, hlo, hhi, [&](int32_t f) {
                table_insert<L>(tab, lgT, f, 1, smin, unweighted, meta, sl);
              });
              if (core_row && hnit > 0)
                for (int32_t p = s_misc[2] + (int32_t)threadIdx.x; p < s_misc[3];
                     p += kGiantNT) {
                  const int32_t f = ci.core_list[p];
                  const int32_t wt = Trow[p];
                  if (wt > 0 && w.r_off[f + 1] - w.r_off[f] >= smin)
                    table_insert<L>(tab, lgT, f, wt, smin, unweighted, meta, sl);
                }
            };
            int32_t at = 0, used = T, total;
            if (list) {
              insert_all(std::true_type{});
#if SLG_GIANT_LIST_SORT
              // Survivors ordered in the survivor-list area, past their slot
              // indices, while the table is cleared: no front region of the
              // table to clear afterwards, two block barriers fewer per bucket.
              __syncthreads();  // inserts done: the list is final
              const int32_t nl = min(*sl.n, sl.cap);
              if (emit && nl <= kGiantListSortMax) {  // uniform
                unsigned long long *lk =
                    reinterpret_cast<unsigned long long *>(sl.slot) + ((nl + 1) >> 1);
                for (int32_t i = threadIdx.x; i < nl; i += kGiantNT)
                  lk[i] = tab[sl.slot[i]] + 1ull;  // the count word holds count - 1
                __syncthreads();  // keys in place; every table and slot read done
                clear_slots<kGiantNT>(tab, T);
                if (threadIdx.x == 0) *sl.n = 0;
                if (a.mode == kStage && out + nl > q4) {  // uniform
                  if (threadIdx.x == 0) raise_error(meta, SLG_ERR_INVALID, kWhereGiant);
                  __syncthreads();
                  return false;
                }
                // each key goes straight to its ranked place in the row's output
                rank_keys<kGiantNT>(lk, nl, [&](int32_t r, unsigned long long x) {
                  const int32_t f = (int32_t)(x >> 32), n = (int32_t)(uint32_t)x;
                  if (a.mode == kDirect) {
                    put(a, base, out + r, e, f, n);
                  } else {
                    tj[out + r] = f;
                    if (!unweighted) tw[out + r] = n;
                  }
                });
                out += nl;
                __syncthreads();  // the keys are read before the next bucket fills the list
                return true;
              }
#endif
              total = table_collect_list<kGiantNT, kGiantQ>(tab, T, sl, emit, &at, &used);
            } else {
              insert_all(std::false_type{});
              __syncthreads();
              total = table_collect<kGiantNT, kGiantSPT>(tab, T, smin, emit, ws, &at, &used);
            }
            return emit_sorted(at, total, used);
          };
          if (!hash_bucket(b0, b1, lo, hi, nit)) break;
        }
        __syncthreads();
        l2_discard(wl, nw);  // the super-chunk's grouped far ends are consumed
        clk_bucket += clock64() - c1;
      }
      if (threadIdx.x == 0) {
        atomicAdd(&meta->giant_cycles[1], (unsigned long long)clk_part);
        atomicAdd(&meta->giant_cycles[2], (unsigned long long)clk_bucket);
      }
    }  // partitioned row
    if (threadIdx.x == 0) *s_base = reserve(a, e, out, kBinGiant);
    __syncthreads();
    if (a.mode == kStage) {
      const long long b = *s_base;
      if (b >= 0)
        for (int32_t i = threadIdx.x; i < out; i += kGiantNT) {
          a.stage_j[b + i] = tj[i];
          if (!unweighted) a.stage_w[b + i] = tw[i];
        }
      __syncthreads();
      l2_discard(tj, out);  // the row's pairs are in the staging area
      if (!unweighted) l2_discard(tw, out);
    }
    if (threadIdx.x == 0 && dense)
      atomicAdd(&meta->giant_cycles[3], (unsigned long long)(clock64() - row_t0));
  }
}

// The first walk also copies the row's far ends (in flattened wedge order) to
// the CTA's part of the giant bin's scratch (free while this kernel runs:
// the giant bin runs after it), so that the second pass reads them in order
// instead of walking the tails again.  buf_stride: ints per CTA (0: none).
#ifndef SLG_SP_GBUF
#define SLG_SP_GBUF 1
#endif
// part: 0 every row of the bin, 1 the rows handed out first (the front of
// the list), 2 the others (the back of the list, on their own ticket).
template <int LGT, int MINB>
__global__ __launch_bounds__(kSpNT, MINB) void k_walk_sparse(
    Walk w, const int32_t *__restrict__ rows, EmitArgs a, int32_t *__restrict__ giant_rows,
    int32_t list_len, int32_t *__restrict__ buf, long long buf_stride, int part) {
  constexpr int kT = 1 << LGT;        // candidate table slots
  constexpr int kSPT = kT / kSpNT;    // table slots per thread
  Meta *meta = a.meta;
  if (meta->err) return;
  extern __shared__ __align__(16) unsigned char smem[];
  long long *s_base = reinterpret_cast<long long *>(smem);
  int32_t *s_ovf = reinterpret_cast<int32_t *>(smem + 8);
  int32_t *s_row = reinterpret_cast<int32_t *>(smem + 12);
  uint32_t *filt = reinterpret_cast<uint32_t *>(smem + 32);
  uint32_t *cand = filt + kSpWords;
  unsigned long long *tab = reinterpret_cast<unsigned long long *>(cand + kSpCWords);
  int32_t *cache = reinterpret_cast<int32_t *>(tab + kT);
  int32_t *s_beg = cache + kSpCache;
  int32_t *s_pref = s_beg + kSpNT;
  int32_t *ws = s_pref + kSpNT + 1;
  const int32_t tid = (int32_t)threadIdx.x;
  // clears the first 2^(lgb - 5) filter words and 2^(lgb - 7) candidate
  // filter words (>= 128 and 32: whole uint4 groups)
  auto clear_filters = [&](int lgb) {
    uint4 *f4 = reinterpret_cast<uint4 *>(filt);
    for (int i = tid; i < (1 << (lgb - 7)); i += kSpNT) f4[i] = make_uint4(0, 0, 0, 0);
    uint4 *c4 = reinterpret_cast<uint4 *>(cand);
    for (int i = tid; i < (1 << (lgb - 9)); i += kSpNT) c4[i] = make_uint4(0, 0, 0, 0);
  };
  clear_filters(kSpLogB);
  for (int i = tid; i < kT; i += kSpNT) tab[i] = kEmpty64;
  const unsigned nrows = (unsigned)meta->rows_bin[kBinSparse];
  const unsigned nhuge = meta->sparse_huge;
  unsigned *ticket = part == 2 ? &meta->sparse_ticket_rest : &meta->sparse_ticket;
  const unsigned t_first = part == 2 ? nhuge : 0u;
  const unsigned t_end = part == 1 ? nhuge : nrows;
  const bool unweighted = a.unweighted != 0;
  const bool emit = a.mode != kCount;
  // SM cycles of the CTA's first thread: row set-up, first walk, second
  // walk, collect and order, emit and clear
  long long cyc[5] = {0, 0, 0, 0, 0};
  for (;;) {
    long long t0 = clock64();
    __syncthreads();  // the previous row's clears done
    if (tid == 0) {
      const unsigned t = t_first + atomicAdd(ticket, 1u);
      *s_ovf = 0;
      *s_row = t >= t_end ? -1 : rows[t < nhuge ? t : list_len - 1 - (t - nhuge)];
    }
    __syncthreads();
    const int32_t e = *s_row;
    if (e < 0) break;
    const int32_t smin = s_of(a.row_s, a.smin, e);
    const int32_t work = a.row_work[e - a.row_begin];
    const int32_t k0 = w.r_off[e], k1 = w.r_off[e + 1];
    const bool cached = work <= kSpCache;
    // the far ends kept in global scratch for the second pass (uniform)
    int32_t *gbuf = (SLG_SP_GBUF && !cached && (long long)work <= buf_stride)
                        ? buf + (long long)blockIdx.x * buf_stride
                        : nullptr;
    int lgb, lgt;
    sp_sizes(work, LGT, &lgb, &lgt);
    const int32_t T = 1 << lgt;
    {
      const long long t1 = clock64();
      cyc[0] += t1 - t0;
      t0 = t1;
    }
    // 1. filter; candidates (a thread's G filter updates are in flight together)
    cta_walk_batched<kSpNT, kSpG>(
        w, k0, k1, s_beg, s_pref, ws, [&](const int32_t(&f)[kSpG], int32_t i0) {
          uint32_t old[kSpG], m[kSpG];
#pragma unroll
          for (int g = 0; g < kSpG; ++g) {
            if (cached && f[g] >= 0) cache[i0 + 32 * g] = f[g];
            if (gbuf && f[g] >= 0) gbuf[i0 + 32 * g] = f[g];
            const uint32_t h = sp_h1(f[g], lgb);
            m[g] = f[g] >= 0 ? 1u << (h & 31) : 0u;
            old[g] = f[g] >= 0 ? atomicOr(filt + (h >> 5), m[g]) : 0u;
          }
#if SLG_SP_DEFER
          int32_t pend[kSpG] = {};
          int np = 0;
#pragma unroll
          for (int g = 0; g < kSpG; ++g) pend_push(pend, np, (old[g] & m[g]) != 0, f[g], g);
#pragma unroll
          for (int q = 0; q < kSpG; ++q) {
            if (!__any_sync(0xffffffffu, q < np)) break;
            if (q < np) sp_candidate(tab, cand, pend[q], s_ovf, lgb, lgt);
          }
#else
#pragma unroll
          for (int g = 0; g < kSpG; ++g)
            if (old[g] & m[g]) sp_candidate(tab, cand, f[g], s_ovf, lgb, lgt);
#endif
        });
    __syncthreads();  // candidates final
    {
      const long long t1 = clock64();
      cyc[1] += t1 - t0;
      t0 = t1;
    }
    if (*s_ovf) {  // uniform: too many candidates for the table
      if (tid == 0) {
        // hand the row to the giant bin (launched after this kernel)
        const unsigned pos = atomicAdd(&meta->giant_rest, 1u);
        giant_rows[list_len - 1 - pos] = e;
        atomicAdd(&meta->rows_bin[kBinGiant], 1ull);
      }
      clear_filters(lgb);
      for (int i = tid; i < T; i += kSpNT) tab[i] = kEmpty64;
      continue;
    }
    // 2. exact counts of the candidates
    // (the deferred slow path, as in the walk below)
    auto count_step = [&](const int32_t(&f)[kSpG]) {
      uint32_t word[kSpG], bit[kSpG];
#pragma unroll
      for (int g = 0; g < kSpG; ++g) {  // the candidate filter, loads in flight together
        const uint32_t c = sp_h2(f[g], lgb);
        bit[g] = 1u << (c & 31);
        word[g] = f[g] >= 0 ? cand[c >> 5] : 0u;
      }
      int32_t pend[kSpG] = {};
      int np = 0;
#pragma unroll
      for (int g = 0; g < kSpG; ++g) pend_push(pend, np, (word[g] & bit[g]) != 0, f[g], g);
#pragma unroll
      for (int q = 0; q < kSpG; ++q) {
        if (!__any_sync(0xffffffffu, q < np)) break;
        if (q < np) sp_count_listed(tab, pend[q], smin, unweighted, lgt);
      }
    };
    if (gbuf) {
      // warp-uniform steps over the copy, 32 consecutive far ends per load
      const int32_t lane = tid & 31;
      for (int32_t b0 = (tid >> 5) * 32 * kSpG; b0 < work; b0 += kSpNT * kSpG) {
        int32_t f[kSpG];
#pragma unroll
        for (int g = 0; g < kSpG; ++g) {
          const int32_t i = b0 + 32 * g + lane;
          f[g] = i < work ? gbuf[i] : -1;
        }
        count_step(f);
      }
      __syncthreads();  // every read of the copy done
      l2_discard(gbuf, work);
    } else if (cached) {
      for (int32_t i = tid; i < work; i += kSpNT)
        sp_count(tab, cand, cache[i], smin, unweighted, lgb, lgt);
    } else {
      cta_walk_batched<kSpNT, kSpG>(
          w, k0, k1, s_beg, s_pref, ws, [&](const int32_t(&f)[kSpG], int32_t) {
#if SLG_SP_DEFER
            uint32_t word[kSpG], bit[kSpG];
#pragma unroll
            for (int g = 0; g < kSpG; ++g) {  // the candidate filter, loads in flight together
              const uint32_t c = sp_h2(f[g], lgb);
              bit[g] = 1u << (c & 31);
              word[g] = f[g] >= 0 ? cand[c >> 5] : 0u;
            }
            int32_t pend[kSpG] = {};
            int np = 0;
#pragma unroll
            for (int g = 0; g < kSpG; ++g) pend_push(pend, np, (word[g] & bit[g]) != 0, f[g], g);
#pragma unroll
            for (int q = 0; q < kSpG; ++q) {
              if (!__any_sync(0xffffffffu, q < np)) break;
              if (q < np) sp_count_listed(tab, pend[q], smin, unweighted, lgt);
            }
#else
#pragma unroll
            for (int g = 0; g < kSpG; ++g)
              if (f[g] >= 0) sp_count(tab, cand, f[g], smin, unweighted, lgb, lgt);
#endif
          });
    }
    __syncthreads();  // counts final
    {
      const long long t1 = clock64();
      cyc[2] += t1 - t0;
      t0 = t1;
    }
    // 3. candidates with count >= s, in ascending f at tab[at, at + n)
    int32_t at = 0, used = T;
    // (ordering n survivors needs 2 n + 32 slots of the table)
    const int32_t n = table_collect<kSpNT, kSPT, (SLG_SP_RUNS != 0)>(
        tab, T, smin, emit, ws, &at, &used, (T - 32) / 2);
    if (n < 0) {  // uniform: hand the row to the giant bin, as for an overflow
      __syncthreads();
      if (tid == 0) {
        const unsigned pos = atomicAdd(&meta->giant_rest, 1u);
        giant_rows[list_len - 1 - pos] = e;
        atomicAdd(&meta->rows_bin[kBinGiant], 1ull);
      }
      clear_filters(lgb);
      for (int i = tid; i < T; i += kSpNT) tab[i] = kEmpty64;
      continue;
    }
    if (tid == 0) *s_base = reserve(a, e, n, kBinSparse);
    __syncthreads();
    {
      const long long t1 = clock64();
      cyc[3] += t1 - t0;
      t0 = t1;
    }
    const long long base = *s_base;
    if (emit && base >= 0)
      for (int32_t i = tid; i < n; i += kSpNT) {
        const unsigned long long x = tab[at + i];
        const int32_t f = (int32_t)(x >> 32), c = (int32_t)(uint32_t)x;
        put(a, base, i, e, f, c);
      }
    clear_filters(lgb);  // nothing reads the filters after the second pass
    table_reset_front<kSpNT>(tab, used);
    cyc[4] += clock64() - t0;
  }
  if (tid == 0)
    for (int q = 0; q < 5; ++q) atomicAdd(&meta->sparse_cycles[q], (unsigned long long)cyc[q]);
}

// --------------------------------------------------------------- launch --

namespace {

using CfgS = CtaCfg<256, 2 * kCtaSMaxWork>;
using CfgL = CtaCfg<256, 2 * kCtaLMaxWork>;
#define K_CTA_S k_walk_cta<256, 2 * kCtaSMaxWork, kBinCtaS, 4>
#define K_CTA_L k_walk_cta<256, 2 * kCtaLMaxWork, kBinCtaL, 3>
#define K_SP_BIG k_walk_sparse<kSpLgT, SLG_SP_MINB>
#define K_SP_SMALL k_walk_sparse<kSpSmallLgT, SLG_SP_SMALL_MINB>

struct Occ {
  int sms = 0, warp_blocks = 0, s_blocks = 0, l_blocks = 0, g_blocks = 0, sp_blocks = 0;
  int sp_small_blocks = 0;
  int dev = -1;
};

Occ &occ_for_device() {
  static Occ occ[64];
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  Occ &o = occ[dev & 63];
  std::lock_guard<std::mutex> lock(mu);
  if (o.dev != dev) {
    cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(K_CTA_S, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CfgS::smem());
    cudaFuncSetAttribute(K_CTA_L, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CfgL::smem());
    cudaFuncSetAttribute(k_walk_giant, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)giant_smem());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.warp_blocks, k_walk_warp, kWarpNT, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.s_blocks, K_CTA_S, 256, CfgS::smem());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.l_blocks, K_CTA_L, 256, CfgL::smem());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.g_blocks, k_walk_giant, kGiantNT,
                                                  giant_smem());
    if (o.g_blocks < 1) o.g_blocks = 1;
    cudaFuncSetAttribute(K_SP_BIG, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sparse_smem(kSpLgT));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.sp_blocks, K_SP_BIG, kSpNT,
                                                  sparse_smem(kSpLgT));
    if (o.sp_blocks < 1) o.sp_blocks = 1;
    cudaFuncSetAttribute(K_SP_SMALL, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sparse_smem(kSpSmallLgT));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.sp_small_blocks, K_SP_SMALL, kSpNT,
                                                  sparse_smem(kSpSmallLgT));
    if (o.sp_small_blocks < 1) o.sp_small_blocks = 1;
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

int sparse_ctas() {
  Occ &o = occ_for_device();
  return o.sms * std::max(o.sp_blocks, SLG_SP_BIG_WORK > 0 ? o.sp_small_blocks : 0);
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
  K_CTA_S<<<o.sms * (o.s_blocks > 0 ? o.s_blocks : 1), 256, CfgS::smem(), st>>>(
      L.w, lists + 1 * stride, L.row_work, L.a);
  ++n;
  if (ev) cudaEventRecord(ev[2], st);
  K_CTA_L<<<o.sms * (o.l_blocks > 0 ? o.l_blocks : 1), 256, CfgL::smem(), st>>>(
      L.w, lists + 2 * stride, L.row_work, L.a);
  ++n;
  if (ev) cudaEventRecord(ev[3], st);
  // the sparse bin before the giant bin: a sparse row whose candidates
  // overflow its table is appended to the giant bin's list
  // the sparse CTAs share the giant bin's scratch out (it holds at least
  // 4 x max(giant, sparse row work) ints per giant CTA)
  auto buf_stride = [&](int ctas) -> long long {
    return L.giant_scratch
               ? (L.giant_stride * (long long)(o.sms * o.g_blocks) / (long long)ctas) & ~31ll
               : 0;
  };
  const int sp_big = o.sms * o.sp_blocks;
  int32_t *giant_list = const_cast<int32_t *>(lists) + 3 * stride;
  K_SP_BIG<<<sp_big, kSpNT, sparse_smem(kSpLgT), st>>>(
      L.w, lists + 4 * stride, L.a, giant_list, (int32_t)stride, L.giant_scratch,
      buf_stride(sp_big), SLG_SP_BIG_WORK > 0 ? 1 : 0);
  ++n;
  if (SLG_SP_BIG_WORK > 0) {
    const int sp_small = o.sms * o.sp_small_blocks;
    K_SP_SMALL<<<sp_small, kSpNT, sparse_smem(kSpSmallLgT), st>>>(
        L.w, lists + 4 * stride, L.a, giant_list, (int32_t)stride, L.giant_scratch,
        buf_stride(sp_small), 2);
    ++n;
  }
  if (ev) cudaEventRecord(ev[4], st);
  if (L.giant_scratch) {
    k_walk_giant<<<o.sms * o.g_blocks, kGiantNT, giant_smem(), st>>>(
        L.w, lists + 3 * stride, L.a, L.giant_scratch, L.giant_stride, L.R, (int32_t)stride);
    ++n;
  }
  if (ev) cudaEventRecord(ev[5], st);
  if (launches) *launches += n;
  return cudaGetLastError();
}

}  // namespace slg
