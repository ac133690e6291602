// Planning kernels of the s-overlap walk: input validation, the CSR->CSC
// position map, the CSC filtered by hyperedge size (degree-based pruning,
// Section IV-C: a hyperedge with |e| < s can be in no pair of L_s), the tail
// of every incidence (strict upper triangle, Section IV-C), and the binning of
// rows by wedge work (the GPU counterpart of the load balancing of
// Section IV-F).
#include <algorithm>

#include "slg_internal.cuh"

namespace slg {

namespace {

constexpr int kValNT = 256;

// One warp per row: offsets monotone inside [0, nnz], ids inside [0, cols),
// every row strictly ascending.  Reports through meta (never traps).
__global__ __launch_bounds__(kValNT) void k_validate(const int32_t *__restrict__ off,
                                                     const int32_t *__restrict__ idx,
                                                     int32_t rows, int32_t cols, int64_t nnz,
                                                     Meta *meta, int32_t where_off,
                                                     int32_t where_ids) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kValNT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kValNT) >> 5;
  if (warp == 0 && lane == 0) {
    if (off[0] != 0 || (int64_t)off[rows] != nnz) raise_error(meta, SLG_ERR_INVALID, where_off);
  }
  for (int64_t r = warp; r < rows; r += nwarps) {
    const int32_t lo = off[r], hi = off[r + 1];
    if (lo < 0 || hi < lo || (int64_t)hi > nnz) {
      if (lane == 0) raise_error(meta, SLG_ERR_INVALID, where_off);
      continue;
    }
    bool bad = false;
    for (int32_t k = lo + lane; k < hi; k += 32) {
      const int32_t x = idx[k];
      if (x < 0 || x >= cols) bad = true;
      if (k > lo && idx[k - 1] >= x) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) raise_error(meta, SLG_ERR_INVALID, where_ids);
  }
}

// One warp per CSR row f: the CSC position of every incidence (v, f), found
// by binary search in the (validated, ascending) column v.  A miss means the
// CSR and CSC are not the same incidence.  With nnz equal on both sides and
// strictly ascending rows, a hit for every incidence makes the map a bijection.
__global__ __launch_bounds__(kValNT) void k_csr2csc(Side s, int32_t *__restrict__ csr2csc,
                                                    Meta *meta) {
  if (meta->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kValNT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kValNT) >> 5;
  for (int64_t f = warp; f < s.R; f += nwarps) {
    const int32_t lo = s.r_off[f], hi = s.r_off[f + 1];
    bool bad = false;
    for (int32_t k = lo + lane; k < hi; k += 32) {
      const int32_t v = s.r_idx[k];
      const int32_t q = find_sorted(s.c_idx, s.c_off[v], s.c_off[v + 1], (int32_t)f);
      if (q < 0) bad = true;
      else csr2csc[k] = q;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) raise_error(meta, SLG_ERR_INVALID, kWhereMismatch);
  }
}

// ------------------------------------------ filtered CSC (reduce-then-scan) --

constexpr int kScanNT = 256;
constexpr int kScanIPT = 16;                    // items per thread
constexpr int kScanTile = kScanNT * kScanIPT;   // 4096 CSC entries per tile

__device__ __forceinline__ int32_t kept(const Side &s, int32_t q, int32_t smin) {
  const int32_t f = __ldg(s.c_idx + q);
  return (__ldg(s.r_off + f + 1) - __ldg(s.r_off + f)) >= s_of(s.row_s, smin, f);
}

__global__ __launch_bounds__(kScanNT) void k_filter_reduce(Side s, int32_t smin,
                                                           int32_t *__restrict__ tile,
                                                           const Meta *meta) {
  if (meta->err) return;
  __shared__ int32_t ws[kScanNT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t c = 0;
#pragma unroll 4
  for (int i = 0; i < kScanIPT; ++i) {
    const int64_t q = base + (int64_t)i * kScanNT + threadIdx.x;
    if (q < s.nnz) c += kept(s, (int32_t)q, smin);
  }
  int32_t total;
  block_inclusive_scan<kScanNT>(c, ws, &total);
  if (threadIdx.x == 0) tile[blockIdx.x] = total;
}

// Exclusive scan of n int32 tile sums in place (one CTA); writes the grand
// total to tile[n] and, if given, to *total_out.
__global__ __launch_bounds__(1024) void k_scan_tiles(int32_t *tile, int32_t n,
                                                     int32_t *total_out, const Meta *meta) {
  if (meta->err) return;
  __shared__ int32_t ws[1024 / 32 + 1];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int32_t base = 0; base < n; base += 1024) {
    const int32_t i = base + threadIdx.x;
    const int32_t x = i < n ? tile[i] : 0;
    int32_t total;
    const int32_t inc = block_inclusive_scan<1024>(x, ws, &total);
    if (i < n) tile[i] = carry + inc - x;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    tile[n] = carry;
    if (total_out) *total_out = carry;
  }
}

// Per tile: qs[q] = number of kept entries before q; kept entries are copied
// to their place in the filtered CSC.  Items are strided by kScanNT inside
// the tile so reads stay coalesced; the scan order is item-major.
__global__ __launch_bounds__(kScanNT) void k_filter_scatter(Side s, int32_t smin,
                                                            const int32_t *__restrict__ tile,
                                                            int32_t *__restrict__ qs,
                                                            int32_t *__restrict__ c_idx_s,
                                                            const Meta *meta) {
  if (meta->err) return;
  __shared__ int32_t ws[kScanNT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t carry = tile[blockIdx.x];
  for (int i = 0; i < kScanIPT; ++i) {
    const int64_t q = base + (int64_t)i * kScanNT + threadIdx.x;
    int32_t k = 0, f = 0;
    if (q < s.nnz) {
      f = __ldg(s.c_idx + q);
      k = (__ldg(s.r_off + f + 1) - __ldg(s.r_off + f)) >= s_of(s.row_s, smin, f);
    }
    int32_t total;
    const int32_t inc = block_inclusive_scan<kScanNT>(k, ws, &total);
    if (q < s.nnz) {
      const int32_t pos = carry + inc - k;
      qs[q] = pos;
      if (k) c_idx_s[pos] = f;
    }
    carry += total;
  }
}

__global__ void k_filter_offsets(Side s, const int32_t *__restrict__ qs,
                                 const int32_t *__restrict__ tile, int32_t ntiles,
                                 int32_t *__restrict__ c_off_s, const Meta *meta) {
  if (meta->err) return;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c > s.C) return;
  const int32_t q = s.c_off[c];
  c_off_s[c] = q < s.nnz ? qs[q] : tile[ntiles];
}

// ---------------------------------------------------- tails, work, bins --

constexpr int kRowsNT = 256;
constexpr int kRowsPerBlock = 64;

__device__ __forceinline__ int bin_of(int32_t work, const Bins &b) {
  if (work <= b.warp) return kBinWarp;
  if (work <= b.ctas) return kBinCtaS;
  if (work <= b.ctal) return kBinCtaL;
  return kBinGiant;
}

// A block handles kRowsPerBlock consecutive rows, one warp per row at a time.
// For each incidence (e, v) of an active row: the filtered position of e in
// column v is qs[csr2csc[k]] (e is kept because |e| >= s), so its tail starts
// one past it.  The row's work is the sum of its tail lengths.  Rows with
// work > 0 are appended to their bin's list (one global atomic per bin and
// block); rows outside the range or inactive get n_e = 0.
__global__ __launch_bounds__(kRowsNT) void k_rows_work(Side s, int32_t smin, int32_t row_begin,
                                                       int32_t row_end,
                                                       const int32_t *__restrict__ csr2csc,
                                                       const int32_t *__restrict__ qs,
                                                       const int32_t *__restrict__ c_off_s,
                                                       const int32_t *__restrict__ c_idx_s,
                                                       CoreInfo core, Bins bins,
                                                       int32_t *__restrict__ tail_beg,
                                                       int32_t *__restrict__ tail_end,
                                                       int32_t *__restrict__ n_e,
                                                       long long *__restrict__ stage_pos,
                                                       int32_t *__restrict__ row_work,
                                                       int32_t *__restrict__ bin_rows,
                                                       Meta *meta) {
  if (meta->err) return;
  __shared__ int32_t s_work[kRowsPerBlock];
  // block maxima of the row work (all rows, giant-bin rows, sparse-bin rows):
  // one global atomicMax each per block instead of one per row
  __shared__ int32_t s_max[3];
  __shared__ int32_t s_act;  // active rows (size >= s) of the block
  __shared__ int32_t s_cnt[kNumBins], s_base[kNumBins];
  __shared__ int32_t s_hcnt[2], s_hbase[2];  // giant / sparse rows handed out first
  __shared__ unsigned long long s_w[kNumBins], s_k[kNumBins];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t r0 = row_begin + blockIdx.x * kRowsPerBlock;
  if (threadIdx.x < kNumBins) {
    s_cnt[threadIdx.x] = 0;
    s_w[threadIdx.x] = 0;
    s_k[threadIdx.x] = 0;
  }
  if (threadIdx.x < 2) s_hcnt[threadIdx.x] = 0;
  if (threadIdx.x < 3) s_max[threadIdx.x] = 0;
  if (threadIdx.x == 0) s_act = 0;
  __syncthreads();
  for (int i = warp; i < kRowsPerBlock; i += kRowsNT / 32) {
    const int32_t e = r0 + i;
    int32_t work = 0;
    if (e < row_end) {
      const int32_t lo = s.r_off[e], hi = s.r_off[e + 1];
      const bool core_row = core.row_rank && core.row_rank[e + 1] != core.row_rank[e];
      const bool active = hi - lo >= s_of(s.row_s, smin, e);
      if (active) {
        for (int32_t k = lo + lane; k < hi; k += 32) {
          const int32_t v = s.r_idx[k];
          int32_t tb, te;
          if (core_row && core.col_rank[v + 1] != core.col_rank[v]) {
            // core row at a core column: its tail skips the core rows (their
            // shared core vertices are counted on the tensor cores)
            const int32_t cv = core.col_rank[v];
            int32_t a = core.x_base + core.x_off[cv], b = core.x_base + core.x_off[cv + 1];
            te = b;
            while (a < b) {  // first entry > e
              const int32_t mid = (a + b) >> 1;
              if (c_idx_s[mid] <= e) a = mid + 1;
              else b = mid;
            }
            tb = a;
          } else {
            tb = qs[csr2csc[k]] + 1;
            te = c_off_s[v + 1];
          }
          tail_beg[k] = tb;
          tail_end[k] = te;
          work += te - tb;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) work += __shfl_xor_sync(0xffffffffu, work, d);
      }
      if (lane == 0) {
        n_e[e - row_begin] = 0;
        stage_pos[e - row_begin] = -1;
        row_work[e - row_begin] = work;
        if (work) atomicMax(&s_max[0], work);
        if (active) atomicAdd(&s_act, 1);
      }
    }
    if (lane == 0) {
      // core rows always go to the giant bin (it adds their tile counts),
      // marked by a negative work entry here
      const bool core_row = e < row_end && core.row_rank && core.row_rank[e + 1] != core.row_rank[e] &&
                            s.r_off[e + 1] - s.r_off[e] >= s_of(s.row_s, smin, e);
      s_work[i] = (e < row_end) ? (core_row ? -1 - work : work) : 0;
    }
  }
  __syncthreads();
  int my_bin = -1, my_slot = 0;
  bool huge = false;
  int32_t my_work = 0;
  if (threadIdx.x < kRowsPerBlock) {
    my_work = s_work[threadIdx.x];
    const bool forced = my_work < 0;
    if (forced) my_work = -1 - my_work;
    if (my_work > 0 || forced) {
      const int32_t e = r0 + threadIdx.x;
      my_bin = forced ? (int)kBinGiant : bin_of(my_work, bins);
      // a row with s >= 2 from bins.bloom up to bins.sparse wedges takes the
      // sparse bin; above the CTA bins only when its far ends are sparse in
      // its span (f in (e, R))
      if (!forced && my_work > bins.bloom && my_work <= bins.sparse &&
          s_of(s.row_s, smin, e) >= 2 &&
          (my_bin != kBinGiant ||
           (long long)my_work * bins.dense < (long long)((s.row_fhi ? s.row_fhi[e] : s.R) - 1 - e)))
        my_bin = kBinSparse;
      if (my_bin == kBinGiant) atomicMax(&s_max[1], my_work);
      if (my_bin == kBinSparse) atomicMax(&s_max[2], my_work);
      huge = (my_bin == kBinGiant && my_work > kGiantHugeWork) ||
             (my_bin == kBinSparse && my_work > kSparseBigWork);
      my_slot = huge ? atomicAdd(&s_hcnt[my_bin == kBinSparse], 1) : atomicAdd(&s_cnt[my_bin], 1);
      atomicAdd(&s_w[my_bin], (unsigned long long)my_work);
      atomicAdd(&s_k[my_bin], (unsigned long long)(s.r_off[e + 1] - s.r_off[e]));
    }
  }
  __syncthreads();
  if (threadIdx.x < kNumBins) {
    const int b = threadIdx.x;
    if (b != kBinGiant && b != kBinSparse) {
      s_base[b] = s_cnt[b] ? (int32_t)atomicAdd(&meta->rows_bin[b], (unsigned long long)s_cnt[b]) : 0;
    } else {
      // the huge rows of the giant and sparse bins fill their list from the
      // front, the others from the back (the kernels hand out the huge ones
      // first); rows_bin counts both
      const int q = b == kBinSparse;
      unsigned *rest = q ? &meta->sparse_rest : &meta->giant_rest;
      unsigned *hge = q ? &meta->sparse_huge : &meta->giant_huge;
      if (s_cnt[b] + s_hcnt[q])
        atomicAdd(&meta->rows_bin[b], (unsigned long long)(s_cnt[b] + s_hcnt[q]));
      s_base[b] = s_cnt[b] ? (int32_t)atomicAdd(rest, (unsigned)s_cnt[b]) : 0;
      s_hbase[q] = s_hcnt[q] ? (int32_t)atomicAdd(hge, (unsigned)s_hcnt[q]) : 0;
    }
    if (s_w[b]) {
      atomicAdd(&meta->wedges_bin[b], s_w[b]);
      atomicAdd(&meta->wedges, s_w[b]);
      atomicAdd(&meta->incid_bin[b], s_k[b]);
    }
  }
  if (threadIdx.x == kNumBins && s_act) atomicAdd(&meta->active, (unsigned long long)s_act);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_max[0]) atomicMax(&meta->max_row_work, s_max[0]);
    if (s_max[1]) atomicMax(&meta->max_giant_work, s_max[1]);
    if (s_max[2]) atomicMax(&meta->max_sparse_work, s_max[2]);
  }
  if (my_bin >= 0) {
    const int64_t len = row_end - row_begin;
    int64_t pos = s_base[my_bin] + my_slot;
    if (huge) pos = s_hbase[my_bin == kBinSparse] + my_slot;
    else if (my_bin == kBinGiant || my_bin == kBinSparse) pos = len - 1 - pos;
    bin_rows[(int64_t)my_bin * len + pos] = r0 + threadIdx.x;
  }
}

inline int grid_for(int64_t items, int per_block, int cap = 1 << 20) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

cudaError_t launch_validate(const Side &s, Meta *meta, cudaStream_t st) {
  const int wpb = kValNT / 32;
  k_validate<<<grid_for(s.R, wpb, 65536), kValNT, 0, st>>>(s.r_off, s.r_idx, s.R, s.C, s.nnz, meta,
                                                          kWhereRowOffsets, kWhereRowIds);
  k_validate<<<grid_for(s.C, wpb, 65536), kValNT, 0, st>>>(s.c_off, s.c_idx, s.C, s.R, s.nnz, meta,
                                                          kWhereColOffsets, kWhereColIds);
  return cudaGetLastError();
}

// inv[map[k]] = k for k < n: the CSR->CSC map of the dual side from that of
// the primal side (the dual's CSR is the primal's CSC and vice versa).
__global__ void k_invert(const int32_t *__restrict__ map, int64_t n, int32_t *__restrict__ inv) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t m = map[k];
    if (m >= 0 && m < n) inv[m] = (int32_t)k;  // a validated map is a permutation
  }
}

cudaError_t launch_invert(const int32_t *map, int64_t n, int32_t *inv, cudaStream_t st) {
  if (n > 0) k_invert<<<(int)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(map, n, inv);
  return cudaGetLastError();
}

cudaError_t launch_csr2csc(const Side &s, int32_t *csr2csc, Meta *meta, cudaStream_t st) {
  k_csr2csc<<<grid_for(s.R, kValNT / 32, 65536), kValNT, 0, st>>>(s, csr2csc, meta);
  return cudaGetLastError();
}

cudaError_t launch_filter(const Side &s, int32_t smin, const Work &w, cudaStream_t st) {
  const int32_t ntiles = (int32_t)((s.nnz + kScanTile - 1) / kScanTile);
  if (ntiles > 0) {
    k_filter_reduce<<<ntiles, kScanNT, 0, st>>>(s, smin, w.tile, w.meta);
  }
  k_scan_tiles<<<1, 1024, 0, st>>>(w.tile, ntiles, &w.meta->kept, w.meta);
  if (ntiles > 0) {
    k_filter_scatter<<<ntiles, kScanNT, 0, st>>>(s, smin, w.tile, w.qs, w.c_idx_s, w.meta);
  }
  k_filter_offsets<<<grid_for((int64_t)s.C + 1, 256), 256, 0, st>>>(s, w.qs, w.tile, ntiles,
                                                                    w.c_off_s, w.meta);
  return cudaGetLastError();
}

cudaError_t launch_rows_work(const Side &s, int32_t smin, int32_t row_begin, int32_t row_end,
                             const Work &w, const CoreInfo &core, const Bins &bins,
                             cudaStream_t st) {
  const int32_t rows = row_end - row_begin;
  if (rows <= 0) return cudaSuccess;
  const int grid = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
  k_rows_work<<<grid, kRowsNT, 0, st>>>(s, smin, row_begin, row_end, w.csr2csc, w.qs, w.c_off_s,
                                        w.c_idx_s, core, bins,
                                        w.tail_beg, w.tail_end, w.n_e, w.stage_pos, w.row_work,
                                        w.bin_rows,
                                        w.meta);
  return cudaGetLastError();
}

}  // namespace slg
