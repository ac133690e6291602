// Degree-ordered relabelling (Section IV-F renumbers the hyperedges by size,
// largest first; the evaluation in Section V finds ascending order faster).
//
// The walk's strict upper triangle charges every pair to its smaller id, so
// the numbering decides which rows carry the wedges: numbered by ascending
// size, the large rows come last and walk only the short tails of the rows
// after them.  The relabelled side is an ordinary side (CSR + CSC, rows
// strictly ascending), so every algorithm runs on it unchanged; its pairs
// are mapped back to the caller's ids, oriented i < j and re-sorted by (i, j)
// afterwards, so the output is the same canonical edge list.
//
//   perm[k] = caller id of relabelled row k  (stable: by size, then by id)
#include "slg_internal.cuh"

namespace slg {

namespace {

constexpr int kNT = 256;

int grid_for(int64_t items, int per_block) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g > 65536) g = 65536;
  return g < 1 ? 1 : (int)g;
}

// keys[r] = size of row r (descending: C - size, sizes being <= C),
// vals[r] = r.
__global__ __launch_bounds__(kNT) void k_rl_keys(int32_t R, int32_t C,
                                                 const int32_t *__restrict__ r_off,
                                                 int descending, uint32_t *__restrict__ keys,
                                                 int32_t *__restrict__ vals) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t r = (int64_t)blockIdx.x * kNT + threadIdx.x; r < R; r += step) {
    const uint32_t size = (uint32_t)(r_off[r + 1] - r_off[r]);
    keys[r] = descending ? (uint32_t)C - size : size;
    vals[r] = (int32_t)r;
  }
}

// sizes[k] = size of row perm[k]; sizes[R] = 0.
__global__ __launch_bounds__(kNT) void k_rl_sizes(int32_t R, const int32_t *__restrict__ r_off,
                                                  const int32_t *__restrict__ perm,
                                                  int32_t *__restrict__ sizes) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t k = (int64_t)blockIdx.x * kNT + threadIdx.x; k <= R; k += step) {
    if (k == R) {
      sizes[R] = 0;
      continue;
    }
    const int32_t r = perm[k];
    sizes[k] = r_off[r + 1] - r_off[r];
  }
}

// One warp per relabelled row: copy its columns, and emit (column, row)
// pairs in relabelled-row order for the stable regrouping by column.
__global__ __launch_bounds__(kNT) void k_rl_rows(int32_t R, const int32_t *__restrict__ r_off,
                                                 const int32_t *__restrict__ r_idx,
                                                 const int32_t *__restrict__ perm,
                                                 const int32_t *__restrict__ r_off2,
                                                 int32_t *__restrict__ r_idx2,
                                                 uint32_t *__restrict__ col_key,
                                                 int32_t *__restrict__ row_val) {
  const int lane = threadIdx.x & 31;
  const int64_t wstep = (int64_t)gridDim.x * (kNT / 32);
  for (int64_t k = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5; k < R; k += wstep) {
    const int32_t r = perm[k];
    const int32_t a = r_off[r], len = r_off[r + 1] - a, b = r_off2[k];
    for (int32_t t = lane; t < len; t += 32) {
      const int32_t v = __ldg(r_idx + a + t);
      r_idx2[b + t] = v;
      col_key[b + t] = (uint32_t)v;
      row_val[b + t] = (int32_t)k;
    }
  }
}

// Pair (a, b) in relabelled ids -> key (min, max) of the caller's ids.
__global__ __launch_bounds__(kNT) void k_rl_pairs(int64_t P, const int32_t *__restrict__ out_i,
                                                  const int32_t *__restrict__ out_j,
                                                  const int32_t *__restrict__ perm, int rbits,
                                                  unsigned long long *__restrict__ keys) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < P; p += step) {
    const uint32_t i = (uint32_t)__ldg(perm + out_i[p]);
    const uint32_t j = (uint32_t)__ldg(perm + out_j[p]);
    const uint32_t lo = i < j ? i : j, hi = i < j ? j : i;
    keys[p] = ((unsigned long long)lo << rbits) | hi;
  }
}

__global__ __launch_bounds__(kNT) void k_rl_unpack(int64_t P,
                                                   const unsigned long long *__restrict__ keys,
                                                   int rbits, int32_t *__restrict__ out_i,
                                                   int32_t *__restrict__ out_j) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  const unsigned long long mask = (1ull << rbits) - 1;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < P; p += step) {
    const unsigned long long k = keys[p];
    out_i[p] = (int32_t)(k >> rbits);
    out_j[p] = (int32_t)(k & mask);
  }
}

int bits_for(int64_t x) {  // bits needed for values in [0, x]
  int b = 0;
  while (b < 63 && (x >> b) != 0) ++b;
  return b;
}

}  // namespace

int relabel_row_bits(int32_t R) { return bits_for(R > 0 ? R - 1 : 0); }

// Relabelled copy of a side: perm [R]; r_off2 [R + 1]; r_idx2, c_idx2 [nnz]
// (the column offsets do not change).  scratch: relabel_scratch_ints ints.
size_t relabel_scratch_ints(int32_t R, int64_t nnz) {
  const int64_t n = nnz > R ? nnz : R;
  // keys, keys_tmp (u32), vals_tmp, sizes, scan tiles, sort histograms
  return (size_t)(3 * n + (int64_t)R + 1 + xscan_tiles((int64_t)R + 1) + 1) +
         radix_sort_scratch_ints(n);
}

cudaError_t launch_relabel(const Side &sd, int descending, int32_t *perm, int32_t *r_off2,
                           int32_t *r_idx2, int32_t *c_idx2, int32_t *scratch, cudaStream_t st,
                           int32_t *launches) {
  const int32_t R = sd.R;
  const int64_t nnz = sd.nnz;
  const int64_t n = nnz > R ? nnz : R;
  uint32_t *keys = reinterpret_cast<uint32_t *>(scratch);
  uint32_t *keys_tmp = keys + n;
  int32_t *vals_tmp = scratch + 2 * n;
  int32_t *sizes = scratch + 3 * n;
  int32_t *tiles = sizes + R + 1;
  int32_t *hist = tiles + xscan_tiles((int64_t)R + 1) + 1;
  cudaError_t e;
  if (R > 0) {
    // 1. rows by size (stable: equal sizes keep ascending caller ids)
    k_rl_keys<<<grid_for(R, kNT), kNT, 0, st>>>(R, sd.C, sd.r_off, descending, keys, perm);
    e = launch_radix_sort(keys, keys_tmp, perm, vals_tmp, R, 0, bits_for(sd.C), hist, st,
                          launches);
    *launches += 1;
    if (e != cudaSuccess) return e;
  }
  // 2. the relabelled CSR offsets
  k_rl_sizes<<<grid_for((int64_t)R + 1, kNT), kNT, 0, st>>>(R, sd.r_off, perm, sizes);
  e = launch_xscan(sizes, r_off2, (int64_t)R + 1, tiles, st);
  if (e != cudaSuccess) return e;
  *launches += 4;
  if (nnz == 0) return cudaGetLastError();
  // 3. relabelled CSR rows, then the CSC: (column, row) pairs produced in
  // row order and sorted stably by column keep every column ascending.
  k_rl_rows<<<grid_for((int64_t)R * 32, kNT), kNT, 0, st>>>(R, sd.r_off, sd.r_idx, perm, r_off2,
                                                            r_idx2, keys, c_idx2);
  *launches += 1;
  e = launch_radix_sort(keys, keys_tmp, c_idx2, vals_tmp, nnz, 0,
                        bits_for(sd.C > 0 ? sd.C - 1 : 0), hist, st, launches);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// Pairs (out_i, out_j, out_w)[0, P) in relabelled ids -> the canonical list
// in caller ids.  keys: 2 P entries; vals: P ints (only when weighted);
// hist: radix_sort_scratch_ints(P).
cudaError_t launch_unrelabel(int64_t P, int32_t R, const int32_t *perm, int32_t *out_i,
                             int32_t *out_j, int32_t *out_w, unsigned long long *keys,
                             int32_t *vals, int32_t *hist, cudaStream_t st, int32_t *launches) {
  if (P <= 0) return cudaSuccess;
  const int rbits = relabel_row_bits(R);
  k_rl_pairs<<<grid_for(P, kNT * 4), kNT, 0, st>>>(P, out_i, out_j, perm, rbits, keys);
  cudaError_t e = launch_radix_sort(keys, keys + P, out_w, out_w ? vals : nullptr, P, 0,
                                    2 * rbits, hist, st, launches);
  if (e != cudaSuccess) return e;
  k_rl_unpack<<<grid_for(P, kNT * 4), kNT, 0, st>>>(P, keys, rbits, out_i, out_j);
  *launches += 2;
  return cudaGetLastError();
}

}  // namespace slg
