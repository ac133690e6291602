// Threshold filter over a canonical edge list: L_s from L_s' for s >= s'.
//
// Section III defines L_s by the overlap threshold alone, so a pair of L_s'
// belongs to L_s exactly when its weight is >= s: L_s is the sub-list of
// L_s' with w >= s, in the same (i, j) order.  One walk at the smallest
// threshold of a sweep therefore answers every larger one.
//
// Stable compaction in three launches: per tile of kTile triples the count
// of kept ones; an exclusive scan of the tile counts (64-bit); per tile a
// block scan of the kept flags, round by round, writing in order.
#include "slg_internal.cuh"

namespace slg {

namespace {

constexpr int kNT = 256;
constexpr int kRounds = 32;
constexpr int64_t kTile = (int64_t)kNT * kRounds;  // 8192 triples

__global__ __launch_bounds__(kNT) void k_keep_count(const int32_t *__restrict__ w, int64_t n,
                                                    int32_t s, long long *__restrict__ tile) {
  __shared__ int32_t ws[kNT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  int32_t c = 0;
  for (int r = 0; r < kRounds; ++r) {
    const int64_t p = base + (int64_t)r * kNT + threadIdx.x;
    if (p < n) c += __ldg(w + p) >= s;
  }
  int32_t total;
  block_inclusive_scan<kNT>(c, ws, &total);
  if (threadIdx.x == 0) tile[blockIdx.x] = total;
}

// Exclusive scan of the tile counts in place; tile[n] = total.
__global__ __launch_bounds__(1024) void k_keep_scan(long long *tile, int64_t n) {
  __shared__ long long ws[1024 / 32 + 1];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b = 0; b < n; b += 1024) {
    const int64_t i = b + threadIdx.x;
    const long long x = i < n ? tile[i] : 0;
    long long total;
    const long long inc = block_inclusive_scan64<1024>(x, ws, &total);
    if (i < n) tile[i] = carry + inc - x;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) tile[n] = carry;
}

__global__ __launch_bounds__(kNT) void k_keep_write(const int32_t *__restrict__ in_i,
                                                    const int32_t *__restrict__ in_j,
                                                    const int32_t *__restrict__ in_w, int64_t n,
                                                    int32_t s, const long long *__restrict__ tile,
                                                    int32_t *__restrict__ out_i,
                                                    int32_t *__restrict__ out_j,
                                                    int32_t *__restrict__ out_w) {
  __shared__ int32_t ws[kNT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  long long pos = tile[blockIdx.x];
  for (int r = 0; r < kRounds; ++r) {
    const int64_t p = base + (int64_t)r * kNT + threadIdx.x;
    const int32_t wt = p < n ? __ldg(in_w + p) : 0;
    const int32_t keep = p < n && wt >= s;
    int32_t total;
    const int32_t inc = block_inclusive_scan<kNT>(keep, ws, &total);
    if (keep) {
      const long long q = pos + inc - 1;
      out_i[q] = __ldg(in_i + p);
      out_j[q] = __ldg(in_j + p);
      if (out_w) out_w[q] = wt;
    }
    pos += total;
    if (base + (int64_t)(r + 1) * kNT >= n) break;  // uniform
  }
}

}  // namespace

int64_t keep_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

cudaError_t launch_keep_count(const int32_t *w, int64_t n, int32_t s, long long *tile,
                              cudaStream_t st) {
  const int64_t nt = keep_tiles(n);
  if (nt > 0) k_keep_count<<<(unsigned)nt, kNT, 0, st>>>(w, n, s, tile);
  k_keep_scan<<<1, 1024, 0, st>>>(tile, nt);
  return cudaGetLastError();
}

cudaError_t launch_keep_write(const int32_t *in_i, const int32_t *in_j, const int32_t *in_w,
                              int64_t n, int32_t s, const long long *tile, int32_t *out_i,
                              int32_t *out_j, int32_t *out_w, cudaStream_t st) {
  const int64_t nt = keep_tiles(n);
  if (nt > 0)
    k_keep_write<<<(unsigned)nt, kNT, 0, st>>>(in_i, in_j, in_w, n, s, tile, out_i, out_j, out_w);
  return cudaGetLastError();
}

}  // namespace slg
