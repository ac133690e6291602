// Dense-core detection and packing for the tensor-core tile path.
//
// The incidence matrix B (rows = hyperedges of the side, columns = its
// vertices) is split into a dense core block B_c = B[R_c, C_c] and the rest.
// Then B·Bᵀ = B_c·B_cᵀ + (the products of the remaining incidences), and for
// a pair of core rows (e, f) the overlap is
//     |e ∩ f| = (B_c·B_cᵀ)[e, f]  +  #{ common vertices outside C_c },
// while for every other pair no core-block product is involved.  So the walk
// skips exactly the wedges e -> v -> f with e, f in R_c and v in C_c, the
// tensor cores compute B_c·B_cᵀ (slg_tc.cu), and the two counts are added
// before the threshold s.
//
// Core selection (degree thresholds): candidate columns have degree >= tau_c,
// candidate rows at least tau_r incidences in them; C_c = the columns holding
// at least max(8, min_density x |rows|) candidate rows, R_c = the rows with at
// least tau_r incidences in C_c.  Both are ranked in ascending id order
// (scans), so the list of core rows is sorted.
#include "slg_internal.cuh"

namespace slg {

namespace {

constexpr int kNT = 256;

// core_col[v] = 1 if deg(v) >= tau_c (C + 1 entries, last 0).
__global__ void k_core_cols(Side s, int32_t tau_c, int32_t *__restrict__ core_col,
                            const Meta *meta) {
  if (meta->err) return;
  const int64_t v = (int64_t)blockIdx.x * kNT + threadIdx.x;
  if (v > s.C) return;
  core_col[v] = (v < s.C && s.c_off[v + 1] - s.c_off[v] >= tau_c) ? 1 : 0;
}

// core_row[e] = 1 if row e has >= tau_r incidences in core columns; counts
// the core incidences of core rows into meta (one warp per row).
__global__ void k_core_rows(Side s, int32_t tau_r, const int32_t *__restrict__ core_col_rank,
                            int32_t *__restrict__ core_row, unsigned long long *nnz_core,
                            const Meta *meta) {
  if (meta->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kNT) >> 5;
  for (int64_t e = gw; e <= s.R; e += nw) {
    int32_t c = 0;
    if (e < s.R) {
      for (int32_t k = s.r_off[e] + lane; k < s.r_off[e + 1]; k += 32) {
        const int32_t v = s.r_idx[k];
        c += core_col_rank[v + 1] - core_col_rank[v];  // 1 if v is a core column
      }
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    }
    if (lane == 0) {
      const int is_core = (e < s.R && c >= tau_r) ? 1 : 0;
      core_row[e] = is_core;
      if (is_core) atomicAdd(nnz_core, (unsigned long long)c);
    }
  }
}

// A[row_rank[e]][col_rank[v]] = 0x38 for every core incidence (e, v).
__global__ void k_core_pack(Side s, const int32_t *__restrict__ row_rank,
                            const int32_t *__restrict__ col_rank, uint8_t *__restrict__ A,
                            int32_t Kp, const Meta *meta) {
  if (meta->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kNT) >> 5;
  for (int64_t e = gw; e < s.R; e += nw) {
    if (row_rank[e + 1] == row_rank[e]) continue;  // not a core row
    const int64_t ri = row_rank[e];
    for (int32_t k = s.r_off[e] + lane; k < s.r_off[e + 1]; k += 32) {
      const int32_t v = s.r_idx[k];
      if (col_rank[v + 1] != col_rank[v]) A[ri * Kp + col_rank[v]] = 0x38;
    }
  }
}

// Core-excluded filtered CSC of every core column v: the entries of
// c_idx_s[c_off_s[v], c_off_s[v+1]) that are not core rows, appended at
// x_base + x_off[cv] (cv = core rank of v).  One warp per core column; the
// order of the column is kept (ballot compaction).
__global__ void k_core_xcsc(int32_t C, const int32_t *__restrict__ col_rank,
                            const int32_t *__restrict__ c_off_s,
                            const int32_t *__restrict__ c_idx_s,
                            const int32_t *__restrict__ row_rank,
                            const int32_t *__restrict__ x_off, int32_t *__restrict__ x_idx,
                            const Meta *meta) {
  if (meta->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kNT) >> 5;
  for (int64_t v = gw; v < C; v += nw) {
    if (col_rank[v + 1] == col_rank[v]) continue;
    int32_t out = x_off[col_rank[v]];
    for (int32_t q0 = c_off_s[v]; q0 < c_off_s[v + 1]; q0 += 32) {
      const int32_t q = q0 + lane;
      int32_t f = 0;
      bool keep = false;
      if (q < c_off_s[v + 1]) {
        f = c_idx_s[q];
        keep = row_rank[f + 1] == row_rank[f];
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) x_idx[out + __popc(bal & ((1u << lane) - 1))] = f;
      out += __popc(bal);
    }
  }
}

// col_cnt[v] += 1 for every incidence (e, v) of a core row e (warp per row).
__global__ void k_core_colcount(Side s, const int32_t *__restrict__ row_rank,
                                int32_t *__restrict__ col_cnt, const Meta *meta) {
  if (meta->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kNT) >> 5;
  for (int64_t e = gw; e < s.R; e += nw) {
    if (row_rank[e + 1] == row_rank[e]) continue;
    for (int32_t k = s.r_off[e] + lane; k < s.r_off[e + 1]; k += 32)
      atomicAdd(col_cnt + s.r_idx[k], 1);
  }
}

// core_col[v] = 1 if column v holds at least tau core rows (C + 1 entries).
__global__ void k_core_cols_refine(int32_t C, const int32_t *__restrict__ col_cnt, int32_t tau,
                                   int32_t *__restrict__ core_col) {
  const int64_t v = (int64_t)blockIdx.x * kNT + threadIdx.x;
  if (v > C) return;
  core_col[v] = (v < C && col_cnt[v] >= tau) ? 1 : 0;
}

// Per core column: its number of non-core entries in the filtered CSC.
__global__ void k_core_xcount(int32_t C, const int32_t *__restrict__ col_rank,
                              const int32_t *__restrict__ c_off_s,
                              const int32_t *__restrict__ c_idx_s,
                              const int32_t *__restrict__ row_rank, int32_t *__restrict__ x_cnt,
                              const Meta *meta) {
  if (meta->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kNT) >> 5;
  for (int64_t v = gw; v < C; v += nw) {
    if (col_rank[v + 1] == col_rank[v]) continue;
    int32_t c = 0;
    for (int32_t q = c_off_s[v] + lane; q < c_off_s[v + 1]; q += 32) {
      const int32_t f = c_idx_s[q];
      c += row_rank[f + 1] == row_rank[f];
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if (lane == 0) x_cnt[col_rank[v]] = c;
  }
}

// ------------------------------------------- generic int32 exclusive scan --
constexpr int kScanIPT = 16;
constexpr int kScanTile = kNT * kScanIPT;

__global__ __launch_bounds__(kNT) void k_xscan_reduce(const int32_t *__restrict__ in, int64_t n,
                                                      int32_t *__restrict__ tile) {
  __shared__ int32_t ws[kNT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t c = 0;
  for (int i = 0; i < kScanIPT; ++i) {
    const int64_t q = base + (int64_t)i * kNT + threadIdx.x;
    if (q < n) c += in[q];
  }
  int32_t total;
  block_inclusive_scan<kNT>(c, ws, &total);
  if (threadIdx.x == 0) tile[blockIdx.x] = total;
}

__global__ __launch_bounds__(1024) void k_xscan_tiles(int32_t *tile, int32_t n) {
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
}

__global__ __launch_bounds__(kNT) void k_xscan_apply(const int32_t *__restrict__ in, int64_t n,
                                                     const int32_t *__restrict__ tile,
                                                     int32_t *__restrict__ out) {
  __shared__ int32_t ws[kNT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int32_t carry = tile[blockIdx.x];
  for (int i = 0; i < kScanIPT; ++i) {
    const int64_t q = base + (int64_t)i * kNT + threadIdx.x;
    const int32_t x = q < n ? in[q] : 0;
    int32_t total;
    const int32_t inc = block_inclusive_scan<kNT>(x, ws, &total);
    if (q < n) out[q] = carry + inc - x;
    carry += total;
  }
}

// core_list[row_rank[e]] = e for every core row (ascending by construction).
__global__ void k_core_list(int32_t R, const int32_t *__restrict__ row_rank,
                            int32_t *__restrict__ core_list) {
  const int64_t e = (int64_t)blockIdx.x * kNT + threadIdx.x;
  if (e < R && row_rank[e + 1] != row_rank[e]) core_list[row_rank[e]] = (int32_t)e;
}

int grid_warps(int64_t items) {
  int64_t g = (items * 32 + kNT - 1) / kNT;
  if (g > 65536) g = 65536;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

int64_t xscan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// out[i] = in[0] + ... + in[i-1] for i < n (in and out may not alias);
// `tile` has room for xscan_tiles(n) ints.  With in[n-1] = 0 the last entry
// is the total.
cudaError_t launch_xscan(const int32_t *in, int32_t *out, int64_t n, int32_t *tile,
                         cudaStream_t st) {
  const int32_t nt = (int32_t)xscan_tiles(n);
  if (nt == 0) return cudaSuccess;
  k_xscan_reduce<<<nt, kNT, 0, st>>>(in, n, tile);
  k_xscan_tiles<<<1, 1024, 0, st>>>(tile, nt);
  k_xscan_apply<<<nt, kNT, 0, st>>>(in, n, tile, out);
  return cudaGetLastError();
}

cudaError_t launch_core_list(int32_t R, const int32_t *row_rank, int32_t *core_list,
                             cudaStream_t st) {
  if (R <= 0) return cudaSuccess;
  k_core_list<<<(R + kNT - 1) / kNT, kNT, 0, st>>>(R, row_rank, core_list);
  return cudaGetLastError();
}

cudaError_t launch_core_cols(const Side &s, int32_t tau_c, int32_t *core_col, const Meta *meta,
                             cudaStream_t st) {
  k_core_cols<<<(int)((s.C + 1 + kNT - 1) / kNT), kNT, 0, st>>>(s, tau_c, core_col, meta);
  return cudaGetLastError();
}

cudaError_t launch_core_rows(const Side &s, int32_t tau_r, const int32_t *col_rank,
                             int32_t *core_row, unsigned long long *nnz_core, const Meta *meta,
                             cudaStream_t st) {
  k_core_rows<<<grid_warps((int64_t)s.R + 1), kNT, 0, st>>>(s, tau_r, col_rank, core_row,
                                                           nnz_core, meta);
  return cudaGetLastError();
}

cudaError_t launch_core_pack(const Side &s, const int32_t *row_rank, const int32_t *col_rank,
                             uint8_t *A, int32_t Kp, const Meta *meta, cudaStream_t st) {
  k_core_pack<<<grid_warps(s.R), kNT, 0, st>>>(s, row_rank, col_rank, A, Kp, meta);
  return cudaGetLastError();
}

cudaError_t launch_core_refine(const Side &s, const int32_t *row_rank, int32_t *col_cnt,
                               int32_t tau, int32_t *core_col, const Meta *meta,
                               cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(col_cnt, 0, sizeof(int32_t) * ((size_t)s.C + 1), st);
  if (e != cudaSuccess) return e;
  k_core_colcount<<<grid_warps(s.R), kNT, 0, st>>>(s, row_rank, col_cnt, meta);
  k_core_cols_refine<<<(int)((s.C + 1 + kNT - 1) / kNT), kNT, 0, st>>>(s.C, col_cnt, tau, core_col);
  return cudaGetLastError();
}

cudaError_t launch_core_xcount(int32_t C, const int32_t *col_rank, const int32_t *c_off_s,
                               const int32_t *c_idx_s, const int32_t *row_rank, int32_t *x_cnt,
                               const Meta *meta, cudaStream_t st) {
  k_core_xcount<<<grid_warps(C), kNT, 0, st>>>(C, col_rank, c_off_s, c_idx_s, row_rank, x_cnt,
                                               meta);
  return cudaGetLastError();
}

cudaError_t launch_core_xcsc(int32_t C, const int32_t *col_rank, const int32_t *c_off_s,
                             const int32_t *c_idx_s, const int32_t *row_rank,
                             const int32_t *x_off, int32_t *x_idx, const Meta *meta,
                             cudaStream_t st) {
  k_core_xcsc<<<grid_warps(C), kNT, 0, st>>>(C, col_rank, c_off_s, c_idx_s, row_rank, x_off,
                                             x_idx, meta);
  return cudaGetLastError();
}

}  // namespace slg
