// Internal declarations of the slg CUDA library (not part of the C ABI).
//
// Terminology.  The side being computed (H, or H* with SLG_DUAL) has R rows
// (its hyperedges) and C columns (its vertices).  CSR = (r_off, r_idx) lists
// the columns of every row, CSC = (c_off, c_idx) the rows of every column;
// both strictly ascending.  A wedge is a path e -> v -> f with v in e and f in
// N(v) (Section IV-B, the two inner loops of Algorithm 2).  Only wedges with
// f > e are walked (the strict upper triangle of Algorithm 3) and only rows
// with |row| >= s take part (degree-based pruning of Algorithm 3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/slg.h"

namespace slg {

constexpr int kWarp = 32;
constexpr int32_t kEmpty = -1;

// Row bins by wedge work (the degree-binned scheduler).  Rows with s >= 2
// from Bins::bloom up to Bins::sparse wedges go to the sparse bin, the ones
// above the CTA bins only when their far ends are sparse in their id span
// (fewer than one wedge per kDenseRatio ids); the other rows above the CTA
// bins go to the giant bin (dense rows, s = 1, dense-core rows).
enum Bin : int {
  kBinWarp = 0, kBinCtaS = 1, kBinCtaL = 2, kBinGiant = 3, kBinSparse = 4, kNumBins = 5
};

// Upper bounds on a row's wedge count for each non-giant bin.  The hash tables
// hold twice the bound, so a row can never fill its table (distinct
// neighbours <= wedges).
#ifndef SLG_WARP_MAX_WORK
#define SLG_WARP_MAX_WORK 128
#endif
constexpr int32_t kWarpMaxWork = SLG_WARP_MAX_WORK;
constexpr int32_t kCtaSMaxWork = 1024;
constexpr int32_t kCtaLMaxWork = 4096;
// Giant rows above this work are handed out first (largest-first order
// bounds the tail of the dynamic schedule by the largest remaining row).
#ifndef SLG_GIANT_HUGE_WORK
#define SLG_GIANT_HUGE_WORK 32768
#endif
constexpr int32_t kGiantHugeWork = SLG_GIANT_HUGE_WORK;
// Sparse rows above this work are handed out first, to the sparse kernel
// with the larger candidate table; the others go to the one with the smaller
// table and one more CTA per SM (0: a single sparse kernel, and no sparse
// row is handed out first).
#ifndef SLG_SP_BIG_WORK
#define SLG_SP_BIG_WORK 8192
#endif
constexpr int32_t kSparseBigWork = SLG_SP_BIG_WORK > 0 ? SLG_SP_BIG_WORK : kGiantHugeWork;
// A row is dense when it has at least one wedge per this many ids of its far
// ends' span (swept: 8 best for the giant bin's dense windows).
#ifndef SLG_DENSE_RATIO
#define SLG_DENSE_RATIO 8
#endif
constexpr int kDenseRatio = SLG_DENSE_RATIO;

// Counters the device writes and the host reads once per call.
struct Meta {
  int32_t err;                         // first slg_status raised on the device
  int32_t err_where;                   // which check raised it
  unsigned long long rows_bin[kNumBins];
  unsigned long long wedges_bin[kNumBins];
  unsigned long long incid_bin[kNumBins];
  unsigned long long pairs_bin[kNumBins];
  unsigned long long wedges;           // W_s
  unsigned long long active;           // rows with size >= s in range
  unsigned long long pairs;            // |L_s| over the row range
  unsigned long long stage_cursor;     // staging allocator
  unsigned long long stage_overflow;   // rows that did not fit the staging
  unsigned int giant_ticket;           // dynamic giant-row scheduling
  unsigned int giant_huge;             // giant rows above kGiantHugeWork (front of the list)
  unsigned int giant_rest;             // the other giant rows (back of the list)
  unsigned int sparse_ticket;          // the same three for the sparse bin
  unsigned int sparse_ticket_rest;     // the small-table sparse kernel's own tickets
  unsigned int sparse_huge;
  unsigned int sparse_rest;
  int32_t max_sparse_work;             // largest work of a sparse-bin row
  int32_t kept;                        // entries of the filtered CSC
  int32_t max_giant_work;              // largest work of a giant-bin row
  unsigned long long nnz_core;         // incidences of the dense core
  int32_t max_row_work;                // largest work of any row
  unsigned long long giant_cycles[4];  // giant bin: SM cycles in walk, partition, buckets
  unsigned long long sparse_cycles[5]; // sparse bin: row set-up, walk, collect, emit, staging
};

// Where a device-side check fired (for error reports).
enum Where : int32_t {
  kWhereNone = 0, kWhereRowOffsets = 1, kWhereRowIds = 2, kWhereColOffsets = 3,
  kWhereColIds = 4, kWhereMismatch = 5, kWhereHash = 6, kWhereGiant = 7, kWhereStage = 8,
};

__device__ __forceinline__ void raise_error(Meta *meta, int32_t status, int32_t where) {
  if (atomicCAS(&meta->err, 0, status) == 0) meta->err_where = where;
}

// ------------------------------------------------------------------ scans --

__device__ __forceinline__ int32_t warp_inclusive_scan(int32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  return x;
}

__device__ __forceinline__ long long warp_inclusive_scan64(long long x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  return x;
}

// Block-wide inclusive scan; `ws` is shared scratch of NT/32 + 1 ints.
// Returns the thread's inclusive prefix, writes the block total to *total.
template <int NT>
__device__ __forceinline__ int32_t block_inclusive_scan(int32_t x, int32_t *ws,
                                                        int32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  int32_t inc = warp_inclusive_scan(x);
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int32_t v = lane < NW ? ws[lane] : 0;
    int32_t vi = warp_inclusive_scan(v);
    if (lane < NW) ws[lane] = vi - v;  // exclusive warp offsets
    if (lane == NW - 1) ws[NW] = vi;
  }
  __syncthreads();
  inc += ws[warp];
  *total = ws[NW];
  __syncthreads();  // ws may be reused right after
  return inc;
}

template <int NT>
__device__ __forceinline__ long long block_inclusive_scan64(long long x, long long *ws,
                                                            long long *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  long long inc = warp_inclusive_scan64(x);
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    long long v = lane < NW ? ws[lane] : 0;
    long long vi = warp_inclusive_scan64(v);
    if (lane < NW) ws[lane] = vi - v;
    if (lane == NW - 1) ws[NW] = vi;
  }
  __syncthreads();
  inc += ws[warp];
  *total = ws[NW];
  __syncthreads();
  return inc;
}

// Position of `key` in the ascending array a[lo, hi), or -1.
__device__ __forceinline__ int32_t find_sorted(const int32_t *__restrict__ a, int32_t lo,
                                               int32_t hi, int32_t key) {
  while (lo < hi) {
    int32_t mid = lo + ((hi - lo) >> 1);
    int32_t x = __ldg(a + mid);
    if (x < key) lo = mid + 1;
    else if (x > key) hi = mid;
    else return mid;
  }
  return -1;
}

// Multiplicative hash onto [0, T) (Fibonacci hashing + fast range).
__device__ __forceinline__ uint32_t hash_slot(int32_t f, uint32_t T) {
  return __umulhi((uint32_t)f * 0x9E3779B1u, T);
}

// --------------------------------------------------------- wedge walking --
//
// The rows's incidences k in [k0, k1) each own a "tail": the entries after the
// row in the filtered CSC of their column, c_idx_s[tail_beg[k], c_off_s[v+1]).
// The union of the tails (as a multiset) is the row's wedge list.  The walkers
// below flatten the tails and hand every wedge's far end f to `fn`, with the
// work of a batch spread evenly over the threads (load-balanced search over
// the prefix sums of the tail lengths) and coalesced reads of c_idx_s.

struct Walk {
  const int32_t *r_off, *r_idx;      // CSR of the side
  const int32_t *c_idx_s;            // far ends: CSC filtered to rows of size >= s
  const int32_t *tail_beg;           // per CSR incidence: its tail [beg, end)
  const int32_t *tail_end;
};

// CTA-wide walker.  Shared scratch: s_beg[NT], s_pref[NT + 1], ws[NT/32 + 1].
// fn(f, i) receives every wedge's far end f and its index i in the row's
// flattened wedge list (0 .. work-1).
//
// Lane layout (the default): a batch's flattened wedges are cut into chunks
// of 32 G; warp w takes chunks w, w + NT/32, ...; in a chunk, lane l takes
// wedges c0 + 32 g + l (g < G), so every warp-wide load of far ends reads
// 32 consecutive wedges (a few tails) and is coalesced.  The chunk's first
// incidence is found by one binary search (the same address in every lane);
// each lane then steps forward over the incidences its wedges cross.
#ifndef SLG_WALK_LANES
#define SLG_WALK_LANES 1
#endif
template <int NT, int G, bool kBatched = false, class Fn>
__device__ __forceinline__ void cta_walk_lanes(const Walk &w, int32_t k0, int32_t k1,
                                               int32_t *s_beg, int32_t *s_pref, int32_t *ws,
                                               Fn &&fn) {
  const int32_t lane = (int32_t)(threadIdx.x & 31);
  int32_t done = 0;  // wedges of earlier batches
  for (int32_t base = k0; base < k1; base += NT) {
    const int32_t k = base + (int32_t)threadIdx.x;
    int32_t b = 0, len = 0;
    if (k < k1) {
      b = __ldg(w.tail_beg + k);
      len = __ldg(w.tail_end + k) - b;
    }
    int32_t total;
    const int32_t inc = block_inclusive_scan<NT>(len, ws, &total);
    s_beg[threadIdx.x] = b;
    s_pref[threadIdx.x + 1] = inc;
    if (threadIdx.x == 0) s_pref[0] = 0;
    __syncthreads();
    for (int32_t c0 = (int32_t)(threadIdx.x >> 5) * 32 * G; c0 < total; c0 += NT * G) {
      int32_t lo = 0, hi = NT;  // invariant: s_pref[lo] <= c0 < s_pref[hi]
      while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (s_pref[mid] <= c0) lo = mid;
        else hi = mid;
      }
      int32_t src[G];
      int32_t j = lo;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int32_t i = c0 + 32 * g + lane;
        src[g] = -1;
        if (i < total) {
          while (s_pref[j + 1] <= i) ++j;
          src[g] = s_beg[j] + (i - s_pref[j]);
        }
      }
      int32_t f[G];
#pragma unroll
      for (int g = 0; g < G; ++g) f[g] = src[g] >= 0 ? __ldg(w.c_idx_s + src[g]) : -1;
      if constexpr (kBatched) {
        fn(f, done + c0 + lane);  // f[g] < 0: no wedge; index of f[g]: + 32 g
      } else {
#pragma unroll
        for (int g = 0; g < G; ++g)
          if (src[g] >= 0) fn(f[g], done + c0 + 32 * g + lane);
      }
    }
    done += total;
    __syncthreads();
  }
}

// The lane-layout walker handing each thread's G far ends of a step to
// fn(f[G], i0) at once (f[g] = -1 where there is no wedge; the index of
// f[g] is i0 + 32 g), so that fn can issue its shared-memory updates for
// all of them before using any result.
template <int NT, int G, class Fn>
__device__ __forceinline__ void cta_walk_batched(const Walk &w, int32_t k0, int32_t k1,
                                                 int32_t *s_beg, int32_t *s_pref, int32_t *ws,
                                                 Fn &&fn) {
  cta_walk_lanes<NT, G, true>(w, k0, k1, s_beg, s_pref, ws, fn);
}

// Thread layout: each thread takes G consecutive wedges per step, found by
// one binary search over the prefix sums.
template <int NT, int G, class Fn>
__device__ __forceinline__ void cta_walk(const Walk &w, int32_t k0, int32_t k1,
                                         int32_t *s_beg, int32_t *s_pref, int32_t *ws,
                                         Fn &&fn) {
#if SLG_WALK_LANES
  cta_walk_lanes<NT, G>(w, k0, k1, s_beg, s_pref, ws, fn);
  return;
#endif
  int32_t done = 0;  // wedges of earlier batches
  for (int32_t base = k0; base < k1; base += NT) {
    const int32_t k = base + (int32_t)threadIdx.x;
    int32_t b = 0, len = 0;
    if (k < k1) {
      b = __ldg(w.tail_beg + k);
      len = __ldg(w.tail_end + k) - b;
    }
    int32_t total;
    const int32_t inc = block_inclusive_scan<NT>(len, ws, &total);
    s_beg[threadIdx.x] = b;
    s_pref[threadIdx.x + 1] = inc;
    if (threadIdx.x == 0) s_pref[0] = 0;
    __syncthreads();
    for (int32_t i0 = (int32_t)threadIdx.x * G; i0 < total; i0 += NT * G) {
      int32_t lo = 0, hi = NT;  // invariant: s_pref[lo] <= i0 < s_pref[hi]
      while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (s_pref[mid] <= i0) lo = mid;
        else hi = mid;
      }
      // positions first, then the G loads (independent, all in flight)
      int32_t src[G];
      int32_t j = lo;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int32_t i = i0 + g;
        src[g] = -1;
        if (i < total) {
          while (s_pref[j + 1] <= i) ++j;
          src[g] = s_beg[j] + (i - s_pref[j]);
        }
      }
      int32_t f[G];
#pragma unroll
      for (int g = 0; g < G; ++g) f[g] = src[g] >= 0 ? __ldg(w.c_idx_s + src[g]) : -1;
#pragma unroll
      for (int g = 0; g < G; ++g)
        if (src[g] >= 0) fn(f[g], done + i0 + g);
    }
    done += total;
    __syncthreads();
  }
}

// ------------------------------------------------------------- launchers --
// All launchers enqueue on `st` and return the first CUDA error, if any.

struct Side {
  int32_t R, C;     // rows (hyperedges of the side), columns (its vertices)
  int64_t nnz;
  const int32_t *r_off, *r_idx, *c_off, *c_idx;
  const int32_t *row_s = nullptr;  // per-row threshold (batched form), else null
  // per-row bound on far ends (batched form: a row's far ends lie below the
  // end of its member's rows), else null: R
  const int32_t *row_fhi = nullptr;
};

// Threshold of row e: its own (batched form) or the call's s.
__device__ __forceinline__ int32_t s_of(const int32_t *row_s, int32_t smin, int32_t e) {
  return row_s ? __ldg(row_s + e) : smin;
}

// Wedge-work thresholds of the bins (runtime; each at most the capacity the
// bin's kernel is compiled for: kWarpMaxWork, kCtaSMaxWork, kCtaLMaxWork).
// `sparse`: sparse rows above the CTA bins up to this work take the sparse
// bin (larger ones hold more repeated far ends per window than its table,
// and the giant bin's partition serves them better); 0 turns the bin off.
// `bloom`: rows with s >= 2 above this work (and at most `sparse`) take the
// sparse bin also when they are dense or fit a CTA bin.
#ifndef SLG_SPARSE_MAX_WORK
#define SLG_SPARSE_MAX_WORK 16384
#endif
#ifndef SLG_BLOOM_MIN_WORK
#define SLG_BLOOM_MIN_WORK 1024
#endif
// `dense`: a row with at least one wedge per `dense` ids of its far ends'
// span is dense (the giant bin counts it in dense windows).
struct Bins {
  int32_t warp = kWarpMaxWork, ctas = kCtaSMaxWork, ctal = kCtaLMaxWork;
  int32_t sparse = SLG_SPARSE_MAX_WORK;
  int32_t bloom = SLG_BLOOM_MIN_WORK;
  int32_t dense = kDenseRatio;
};

// Dense core for the tensor-core tile path (all null / 0 when unused).
// Core rows form an ascending list; row_rank / col_rank are exclusive scans
// of the core flags (rank[x+1] != rank[x] marks a core member).  For core
// columns, the entries of the filtered CSC that are not core rows are stored
// at c_idx_s[x_base + x_off[rank] .. x_base + x_off[rank + 1]).  T holds the
// tile counts |e ∩ f ∩ C_c| of core rows, row-major with stride Mp.
struct CoreInfo {
  const int32_t *row_rank, *col_rank;
  const int32_t *x_off;
  int32_t x_base;
  const int32_t *core_list;
  int32_t n_core;
  const int32_t *T;
  int32_t Mp;
};

// Per-call device buffers (carved out of one pool allocation).
struct Work {
  int32_t *csr2csc;    // [nnz] CSC position of every CSR incidence
  int32_t *qs;         // [nnz + 1] exclusive scan of "row of this CSC entry kept"
  int32_t *c_idx_s;    // [nnz] filtered CSC ids
  int32_t *c_off_s;    // [C + 1] filtered CSC offsets
  int32_t *tail_beg;   // [nnz] tail of each incidence: [tail_beg, tail_end)
  int32_t *tail_end;   // [nnz]
  int32_t *tile;       // [ntiles + 1] scan scratch
  int32_t *bin_rows;   // [kNumBins][R] row lists
  int32_t *n_e;        // [R] pairs per row
  int32_t *row_work;   // [R] wedges per row
  long long *stage_pos;// [R] staging offset per row, -1 = not staged
  long long *row_ptr;  // [R + 1] output offsets (relative to row_begin)
  long long *tile64;   // [ntiles64 + 1]
  int32_t *stage_j, *stage_w;  // [stage_cap]
  long long stage_cap;
  Meta *meta;
};

cudaError_t launch_validate(const Side &s, Meta *meta, cudaStream_t st);
cudaError_t launch_csr2csc(const Side &s, int32_t *csr2csc, Meta *meta, cudaStream_t st);
// inv[map[k]] = k (k < n): a permutation's inverse.
cudaError_t launch_invert(const int32_t *map, int64_t n, int32_t *inv, cudaStream_t st);
cudaError_t launch_filter(const Side &s, int32_t smin, const Work &w, cudaStream_t st);
cudaError_t launch_rows_work(const Side &s, int32_t smin, int32_t row_begin, int32_t row_end,
                             const Work &w, const CoreInfo &core, const Bins &bins,
                             cudaStream_t st);

// Dense-core detection / packing (slg_core.cu).
int64_t xscan_tiles(int64_t n);
cudaError_t launch_xscan(const int32_t *in, int32_t *out, int64_t n, int32_t *tile,
                         cudaStream_t st);
cudaError_t launch_core_cols(const Side &s, int32_t tau_c, int32_t *core_col, const Meta *meta,
                             cudaStream_t st);
cudaError_t launch_core_rows(const Side &s, int32_t tau_r, const int32_t *col_rank,
                             int32_t *core_row, unsigned long long *nnz_core, const Meta *meta,
                             cudaStream_t st);
cudaError_t launch_core_list(int32_t R, const int32_t *row_rank, int32_t *core_list,
                             cudaStream_t st);
cudaError_t launch_core_refine(const Side &s, const int32_t *row_rank, int32_t *col_cnt,
                               int32_t tau, int32_t *core_col, const Meta *meta,
                               cudaStream_t st);
cudaError_t launch_core_pack(const Side &s, const int32_t *row_rank, const int32_t *col_rank,
                             uint8_t *A, int32_t Kp, const Meta *meta, cudaStream_t st);
cudaError_t launch_core_xcount(int32_t C, const int32_t *col_rank, const int32_t *c_off_s,
                               const int32_t *c_idx_s, const int32_t *row_rank, int32_t *x_cnt,
                               const Meta *meta, cudaStream_t st);
cudaError_t launch_core_xcsc(int32_t C, const int32_t *col_rank, const int32_t *c_off_s,
                             const int32_t *c_idx_s, const int32_t *row_rank,
                             const int32_t *x_off, int32_t *x_idx, const Meta *meta,
                             cudaStream_t st);
// Output modes of the walk: COUNT (pairs per row only), STAGE (each row's
// sorted pairs appended to a staging area at an atomically reserved offset),
// DIRECT (written to their final place; row_ptr known).
enum Mode : int { kCount = 0, kStage = 1, kDirect = 2 };

struct EmitArgs {
  int mode;
  int unweighted;
  const int32_t *row_s;               // per-row threshold, or null: smin
  const int32_t *row_fhi;             // per-row far-end bound, or null: R
  int32_t dense_ratio;                // Bins::dense
  int full_rows;                      // 1: tails are whole columns, far ends in [0, R)
  const int32_t *row_work;            // [rows] wedges per row (giant bin)
  CoreInfo core;                      // dense core (tile counts added by the giant bin)
  int32_t smin;
  int32_t row_begin;
  int32_t *n_e;                       // [rows] pairs per row
  long long *stage_pos;               // [rows] staging offset, -1 = none
  int32_t *stage_j, *stage_w;         // STAGE
  long long stage_cap;
  const long long *row_ptr;           // DIRECT
  int32_t *out_i, *out_j, *out_w;     // DIRECT
  Meta *meta;
};

struct WalkLaunch {
  Walk w;
  EmitArgs a;
  const int32_t *bin_rows;  // [kNumBins][rows] row lists
  const int32_t *row_work;  // [rows] wedges per row
  int32_t rows;             // rows in the range (list stride)
  int32_t *giant_scratch;   // [giant_ctas][4 * max giant work] wedge ends + pairs
  long long giant_stride;   // ints per giant CTA
  int32_t R;                // rows of the side (far ends lie in [0, R))
};

// CTAs of the giant kernel (two per SM) and of the sparse kernel.
int giant_ctas();
int sparse_ctas();
// The largest side (rows) a build supports: row ids and the giant bin's
// super-chunk bounds stay below 2^31.
constexpr int32_t kMaxRows = (int32_t)((1u << 31) - (1u << 23));
// The largest id space of slg_components (its bounded union-find loop).
constexpr int32_t kComponentsMaxR = 1 << 24;

// ev (optional): kNumBins + 1 events recorded before the first and after
// every bin kernel, in launch order (warp, CTA small, CTA large, sparse,
// giant); bin b runs from ev[kWalkEv[b]] to ev[kWalkEv[b] + 1].
constexpr int kWalkEv[kNumBins] = {0, 1, 2, 4, 3};
cudaError_t launch_walk(const WalkLaunch &L, cudaStream_t st, int32_t *launches,
                        cudaEvent_t *ev = nullptr);
cudaError_t launch_row_scan(int32_t rows, const Work &w, cudaStream_t st);
// The device Meta into host memory the device can address (mapped pinned
// memory), by a kernel: no copy engine involved.
cudaError_t launch_meta_copy(const Meta *src, Meta *dst, cudaStream_t st);
// w16[i] = w[i] (i < n); *bad = 1 if a weight is above 65,535.
cudaError_t launch_pack_w16(const int32_t *w, int64_t n, uint16_t *w16, int32_t *bad,
                            cudaStream_t st);
// out_cap: entries of the output arrays (a row beyond them raises an error).
cudaError_t launch_gather(int32_t row_begin, int32_t rows, const Work &w, int32_t *out_i,
                          int32_t *out_j, int32_t *out_w, int unweighted, long long out_cap,
                          cudaStream_t st);

// Batched form (slg_plan.cu): union of many hypergraphs.
struct BatchGraph {            // one member, device pointers
  const int32_t *e_off, *e_idx, *v_off, *v_idx;
  int32_t m, n;
  int64_t nnz;
  int32_t e_base, v_base;      // id offsets in the union
  int64_t k_base;              // incidence offset in the union
  int32_t s;
};
cudaError_t launch_concat(const BatchGraph *g, int32_t count, int32_t max_len, int32_t *e_off,
                          int32_t *e_idx, int32_t *v_off, int32_t *v_idx, int32_t *row_s_e,
                          int32_t *row_s_v, int32_t *row_fhi_e, int32_t *row_fhi_v,
                          cudaStream_t st);
cudaError_t launch_localize(int32_t *out_i, int32_t *out_j, long long pairs,
                            const int32_t *row_base, int32_t count, const long long *row_ptr,
                            long long *offsets, cudaStream_t st);

int giant_ctas_for_device();

// Plain per-hyperedge kernel (comparison): `warps` warps, each with R_pad
// counters in `scratch` and R_pad/1024 bitmap words in `summ`, all zero.
cudaError_t launch_plain(const Side &sd, int32_t smin, int32_t row_begin, int32_t row_end,
                         const EmitArgs &a, int32_t *scratch, uint32_t *summ, int32_t R_pad,
                         int32_t warps, cudaStream_t st);

// Dense-core tile path (tcgen05): C = A·Aᵀ on the upper-triangle 128 x 128
// tiles of an Mp x Kp byte matrix A (0x38 = 1.0).  `tasks` holds room for
// nt (nt + 1) / 2 tile pairs (nt = Mp / 128), `err` one device int.
cudaError_t launch_tile_overlap(const uint8_t *A, int32_t Mp, int32_t Kp, int32_t *C,
                                void *tasks, int32_t *err, cudaStream_t st);
size_t tile_overlap_smem();

// Stable LSD radix sort (slg_sort.cu) by bits [begin_bit, end_bit) of the
// keys, values alongside (vals may be null); tmp buffers of n entries,
// hist of radix_sort_scratch_ints(n) ints; the result ends in keys / vals.
// `launches` (optional) counts the kernels launched.
size_t radix_sort_scratch_ints(int64_t n);
cudaError_t launch_radix_sort(unsigned long long *keys, unsigned long long *keys_tmp,
                              int32_t *vals, int32_t *vals_tmp, int64_t n, int begin_bit,
                              int end_bit, int32_t *hist, cudaStream_t st,
                              int32_t *launches = nullptr);
cudaError_t launch_radix_sort(uint32_t *keys, uint32_t *keys_tmp, int32_t *vals,
                              int32_t *vals_tmp, int64_t n, int begin_bit, int end_bit,
                              int32_t *hist, cudaStream_t st, int32_t *launches = nullptr);

// Degree-ordered relabelling (slg_relabel.cu).
int relabel_row_bits(int32_t R);
size_t relabel_scratch_ints(int32_t R, int64_t nnz);
cudaError_t launch_relabel(const Side &sd, int descending, int32_t *perm, int32_t *r_off2,
                           int32_t *r_idx2, int32_t *c_idx2, int32_t *scratch, cudaStream_t st,
                           int32_t *launches);
cudaError_t launch_unrelabel(int64_t P, int32_t R, const int32_t *perm, int32_t *out_i,
                             int32_t *out_j, int32_t *out_w, unsigned long long *keys,
                             int32_t *vals, int32_t *hist, cudaStream_t st, int32_t *launches);

// Threshold filter of a canonical edge list (slg_sweep.cu): tile counts of
// the triples with w >= s and their exclusive scan in `tile` (keep_tiles(n)
// + 1 entries, tile[keep_tiles(n)] = total), then the ordered compaction.
int64_t keep_tiles(int64_t n);
cudaError_t launch_keep_count(const int32_t *w, int64_t n, int32_t s, long long *tile,
                              cudaStream_t st);
cudaError_t launch_keep_write(const int32_t *in_i, const int32_t *in_j, const int32_t *in_w,
                              int64_t n, int32_t s, const long long *tile, int32_t *out_i,
                              int32_t *out_j, int32_t *out_w, cudaStream_t st);

// After the edge list (slg_post.cu): pair checks, ID squeezing, adjacency,
// components.
cudaError_t launch_check_pairs(const int32_t *a, const int32_t *b, int64_t n, int32_t R,
                               int canonical, int32_t *err, cudaStream_t st);
cudaError_t launch_mark(const int32_t *a, const int32_t *b, int64_t n, int32_t *mark,
                        cudaStream_t st);
cudaError_t launch_squeeze(const int32_t *a, const int32_t *b, int64_t n, int32_t R,
                           const int32_t *mark, const int32_t *rank, int32_t *oa, int32_t *ob,
                           int32_t *old_of_new, cudaStream_t st);
cudaError_t launch_adjacency_offsets(const int32_t *a, const int32_t *b, int64_t n, int32_t V,
                                     int32_t *up, int32_t *lo, long long *off, cudaStream_t st);
cudaError_t launch_adjacency_fill(const int32_t *a, const int32_t *b, const int32_t *w,
                                  int64_t n, int32_t V, const long long *off, const int32_t *lo,
                                  long long *first, long long *lfirst, uint32_t *keys,
                                  uint32_t *keys_tmp, int32_t *pos, int32_t *pos_tmp,
                                  int32_t *hist, int32_t *adj, int32_t *adj_w, cudaStream_t st);
cudaError_t launch_components(const int32_t *a, const int32_t *b, int64_t n, int32_t R,
                              int32_t *labels, const int32_t *mark, unsigned long long *n_comp,
                              int32_t *err, cudaStream_t st);

// Filtered SpGEMM comparison: full-column tails / per-row work, filtration.
cudaError_t launch_rows_full(const Side &sd, int32_t row_begin, int32_t row_end,
                             int32_t list_base, int32_t *tail_beg, int32_t *tail_end,
                             int32_t *work_out,
                             int32_t *n_e, long long *stage_pos, int32_t *bin_rows,
                             int32_t list_stride, Meta *meta, cudaStream_t st);
cudaError_t launch_filter_count(int32_t row_begin, int32_t row_end, int32_t list_base,
                                const Work &w, int32_t smin, int32_t *kept, cudaStream_t st);
cudaError_t launch_filter_write(int32_t row_begin, int32_t row_end, int32_t list_base,
                                const Work &w, int32_t smin, const long long *row_ptr,
                                long long out_base, int unweighted, int32_t *out_i,
                                int32_t *out_j, int32_t *out_w, cudaStream_t st);

}  // namespace slg
