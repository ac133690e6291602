// Filtered SpGEMM comparison path (SLG_ALGO_SPGEMM), the linear-algebra form
// of Section IV-D: materialise C = B·Bᵀ (B the hyperedge-by-vertex 0/1
// incidence) row by row with Gustavson's method -- row i of C is the sum of
// the columns N(v), v in e_i, over the WHOLE column (both triangles and the
// diagonal, no size pruning) -- and only afterwards apply the filtration
// j > i, C_ij >= s.  The row products reuse the binned counting kernels with
// full columns as tails and threshold 1; rows are processed in chunks whose
// product fits a memory budget.
#include "slg_internal.cuh"

namespace slg {

namespace {

constexpr int kNT = 256;
constexpr int kRowsPerBlock = 64;

__device__ __forceinline__ int bin_of_full(int32_t work) {
  if (work <= kWarpMaxWork) return kBinWarp;
  if (work <= kCtaSMaxWork) return kBinCtaS;
  if (work <= kCtaLMaxWork) return kBinCtaL;
  return kBinGiant;
}

// Per row: tails are the whole columns; work = sum of column lengths.
// Writes work[] when `work_out` is given, else bins the rows.
__global__ __launch_bounds__(kNT) void k_rows_full(Side s, int32_t row_begin, int32_t row_end,
                                                   int32_t list_base,
                                                   int32_t *__restrict__ tail_beg,
                                                   int32_t *__restrict__ tail_end,
                                                   int32_t *__restrict__ work_out,
                                                   int32_t *__restrict__ n_e,
                                                   long long *__restrict__ stage_pos,
                                                   int32_t *__restrict__ bin_rows,
                                                   int32_t list_stride, Meta *meta) {
  if (meta->err) return;
  __shared__ int32_t s_work[kRowsPerBlock];
  __shared__ int32_t s_cnt[kNumBins], s_base[kNumBins];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t r0 = row_begin + blockIdx.x * kRowsPerBlock;
  if (threadIdx.x < kNumBins) s_cnt[threadIdx.x] = 0;
  for (int i = warp; i < kRowsPerBlock; i += kNT / 32) {
    const int32_t e = r0 + i;
    int32_t work = 0;
    if (e < row_end) {
      const int32_t lo = s.r_off[e], hi = s.r_off[e + 1];
      for (int32_t k = lo + lane; k < hi; k += 32) {
        const int32_t v = s.r_idx[k];
        const int32_t cb = s.c_off[v], ce = s.c_off[v + 1];
        if (bin_rows) {
          tail_beg[k] = cb;
          tail_end[k] = ce;
        }
        work += ce - cb;
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) work += __shfl_xor_sync(0xffffffffu, work, d);
      if (lane == 0) {
        if (work_out) work_out[e - list_base] = work;
        if (bin_rows) {
          n_e[e - list_base] = 0;
          stage_pos[e - list_base] = -1;
        }
      }
    }
    if (lane == 0) s_work[i] = (e < row_end) ? work : 0;
  }
  if (!bin_rows) return;
  __syncthreads();
  int my_bin = -1, my_slot = 0;
  if (threadIdx.x < kRowsPerBlock && s_work[threadIdx.x] > 0) {
    my_bin = bin_of_full(s_work[threadIdx.x]);
    my_slot = atomicAdd(&s_cnt[my_bin], 1);
    if (my_bin == kBinGiant) atomicMax(&meta->max_giant_work, s_work[threadIdx.x]);
  }
  __syncthreads();
  if (threadIdx.x < kNumBins && s_cnt[threadIdx.x])
    s_base[threadIdx.x] =
        (int32_t)atomicAdd(&meta->rows_bin[threadIdx.x], (unsigned long long)s_cnt[threadIdx.x]);
  __syncthreads();
  if (my_bin >= 0) {
    // giant rows fill their list from the back: k_walk_giant hands out the
    // rows at its front (none here) first, then the back ones
    int64_t pos = s_base[my_bin] + my_slot;
    if (my_bin == kBinGiant) pos = list_stride - 1 - pos;
    bin_rows[(int64_t)my_bin * list_stride + pos] = r0 + threadIdx.x;
  }
}

// Filtration, count: entries of product row e with j > e and value >= s.
__global__ __launch_bounds__(kNT) void k_filter_count(int32_t row_begin, int32_t row_end,
                                                      int32_t list_base,
                                                      const int32_t *__restrict__ n_e,
                                                      const long long *__restrict__ stage_pos,
                                                      const int32_t *__restrict__ stage_j,
                                                      const int32_t *__restrict__ stage_w,
                                                      int32_t smin, int32_t *__restrict__ kept,
                                                      const Meta *meta) {
  if (meta->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kNT) >> 5;
  for (int64_t e = row_begin + gw; e < row_end; e += nw) {
    const int32_t r = (int32_t)(e - list_base);
    const int32_t n = n_e[r];
    const long long b = stage_pos[r];
    int32_t c = 0;
    if (b >= 0)
      for (int32_t t = lane; t < n; t += 32)
        c += (stage_j[b + t] > e) & (stage_w[b + t] >= smin);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if (lane == 0) kept[e - row_begin] = c;
  }
}

// Filtration, write: kept entries in order to out + base + row_ptr[r].
__global__ __launch_bounds__(kNT) void k_filter_write(int32_t row_begin, int32_t row_end,
                                                      int32_t list_base,
                                                      const int32_t *__restrict__ n_e,
                                                      const long long *__restrict__ stage_pos,
                                                      const int32_t *__restrict__ stage_j,
                                                      const int32_t *__restrict__ stage_w,
                                                      int32_t smin,
                                                      const long long *__restrict__ row_ptr,
                                                      long long out_base, int unweighted,
                                                      int32_t *__restrict__ out_i,
                                                      int32_t *__restrict__ out_j,
                                                      int32_t *__restrict__ out_w,
                                                      const Meta *meta) {
  if (meta->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kNT) >> 5;
  for (int64_t e = row_begin + gw; e < row_end; e += nw) {
    const int32_t r = (int32_t)(e - list_base);
    const int32_t n = n_e[r];
    const long long b = stage_pos[r];
    if (b < 0) continue;
    long long o = out_base + row_ptr[e - row_begin];
    for (int32_t t0 = 0; t0 < n; t0 += 32) {
      const int32_t t = t0 + lane;
      int32_t j = 0, w = 0;
      bool keep = false;
      if (t < n) {
        j = stage_j[b + t];
        w = stage_w[b + t];
        keep = (j > e) && (w >= smin);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const long long p = o + __popc(bal & ((1u << lane) - 1));
        out_i[p] = (int32_t)e;
        out_j[p] = j;
        if (!unweighted) out_w[p] = w;
      }
      o += __popc(bal);
    }
  }
}

int grid_rows(int32_t rows) {
  int g = (rows + kRowsPerBlock - 1) / kRowsPerBlock;
  return g < 1 ? 1 : g;
}

int grid_warps(int32_t rows) {
  int64_t g = ((int64_t)rows * 32 + kNT - 1) / kNT;
  if (g > 65536) g = 65536;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t launch_rows_full(const Side &sd, int32_t row_begin, int32_t row_end,
                             int32_t list_base, int32_t *tail_beg, int32_t *tail_end,
                             int32_t *work_out,
                             int32_t *n_e, long long *stage_pos, int32_t *bin_rows,
                             int32_t list_stride, Meta *meta, cudaStream_t st) {
  if (row_end <= row_begin) return cudaSuccess;
  k_rows_full<<<grid_rows(row_end - row_begin), kNT, 0, st>>>(sd, row_begin, row_end, list_base,
                                                              tail_beg, tail_end, work_out, n_e,
                                                              stage_pos,
                                                              bin_rows, list_stride, meta);
  return cudaGetLastError();
}

cudaError_t launch_filter_count(int32_t row_begin, int32_t row_end, int32_t list_base,
                                const Work &w, int32_t smin, int32_t *kept, cudaStream_t st) {
  if (row_end <= row_begin) return cudaSuccess;
  k_filter_count<<<grid_warps(row_end - row_begin), kNT, 0, st>>>(
      row_begin, row_end, list_base, w.n_e, w.stage_pos, w.stage_j, w.stage_w, smin, kept, w.meta);
  return cudaGetLastError();
}

cudaError_t launch_filter_write(int32_t row_begin, int32_t row_end, int32_t list_base,
                                const Work &w, int32_t smin, const long long *row_ptr,
                                long long out_base, int unweighted, int32_t *out_i,
                                int32_t *out_j, int32_t *out_w, cudaStream_t st) {
  if (row_end <= row_begin) return cudaSuccess;
  k_filter_write<<<grid_warps(row_end - row_begin), kNT, 0, st>>>(
      row_begin, row_end, list_base, w.n_e, w.stage_pos, w.stage_j, w.stage_w, smin, row_ptr,
      out_base, unweighted, out_i, out_j, out_w, w.meta);
  return cudaGetLastError();
}

}  // namespace slg
