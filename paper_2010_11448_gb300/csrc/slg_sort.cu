// Stable LSD radix sort of 32- or 64-bit keys with optional 32-bit values,
// used by the degree-ordered relabelling (SLG_RELABEL_*): ordering rows by
// size, regrouping the relabelled incidences by column and restoring the
// caller's (i, j) order of the output.
//
// One pass per 8-bit digit, three kernels per pass (no spin-waits):
//   1. per tile of kTile keys: digit histogram -> hist[digit * ntiles + tile];
//   2. exclusive scan of hist in (digit, tile) order (launch_xscan);
//   3. per tile: each warp ranks its contiguous chunk in order, 32 keys at a
//      time (__match_any_sync on the digit), and scatters stably to
//      hist[digit][tile] + (keys of that digit before it in the tile).
#include "slg_internal.cuh"

namespace slg {

namespace {

constexpr int kSortNT = 256;
constexpr int kSortIPT = 16;
constexpr int kSortTile = kSortNT * kSortIPT;      // 4096 keys per tile
constexpr int kSortWarps = kSortNT / 32;
constexpr int kChunk = kSortTile / kSortWarps;     // 512 keys per warp, in order

template <class K>
__global__ __launch_bounds__(kSortNT) void k_sort_hist(const K *__restrict__ keys, int64_t n,
                                                       int shift, int32_t ntiles,
                                                       int32_t *__restrict__ hist) {
  __shared__ int32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int i = 0; i < kSortIPT; ++i) {
    const int64_t q = base + (int64_t)i * kSortNT + threadIdx.x;
    if (q < n) atomicAdd(h + ((keys[q] >> shift) & 0xFF), 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

template <class K>
__global__ __launch_bounds__(kSortNT) void k_sort_scatter(
    const K *__restrict__ keys, const int32_t *__restrict__ vals, int64_t n, int shift,
    int32_t ntiles, const int32_t *__restrict__ hist, K *__restrict__ keys_out,
    int32_t *__restrict__ vals_out) {
  __shared__ int32_t cnt[kSortWarps][256];  // per warp: its keys per digit, then running
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kSortWarps * 256; d += kSortNT) (&cnt[0][0])[d] = 0;
  __syncthreads();
  const int64_t chunk0 = (int64_t)blockIdx.x * kSortTile + (int64_t)wq * kChunk;
  // 1. per-warp digit counts of its chunk
  for (int i = lane; i < kChunk; i += 32) {
    const int64_t q = chunk0 + i;
    if (q < n) atomicAdd(&cnt[wq][(keys[q] >> shift) & 0xFF], 1);
  }
  __syncthreads();
  // 2. warp offsets per digit: tile offset + keys of earlier warps
  {
    const int d = threadIdx.x;  // kSortNT == 256 digits
    int32_t run = hist[(int64_t)d * ntiles + blockIdx.x];
    for (int w = 0; w < kSortWarps; ++w) {
      const int32_t c = cnt[w][d];
      cnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  // 3. in-order ranking, 32 keys at a time
  for (int i0 = 0; i0 < kChunk; i0 += 32) {
    const int64_t q = chunk0 + i0 + lane;
    const bool live = q < n;
    const K k = live ? keys[q] : K(0);
    const int d = live ? (int)((k >> shift) & 0xFF) : 256 + lane;  // dead lanes: unique
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (live) {
      const int32_t dst = cnt[wq][d] + __popc(peers & ((1u << lane) - 1));
      keys_out[dst] = k;
      if (vals) vals_out[dst] = vals[q];
    }
    __syncwarp();
    if (live && lane == 31 - __clz(peers)) cnt[wq][d] += __popc(peers);  // highest peer
    __syncwarp();
  }
}

}  // namespace

// Histogram, its scan and the scan's tile sums.
size_t radix_sort_scratch_ints(int64_t n) {
  int64_t ntiles = (n + kSortTile - 1) / kSortTile;
  if (ntiles < 1) ntiles = 1;
  return (size_t)(2 * 256 * ntiles + xscan_tiles(256 * ntiles) + 1);
}

namespace {

template <class K>
cudaError_t radix_sort(K *keys, K *keys_tmp, int32_t *vals, int32_t *vals_tmp, int64_t n,
                       int begin_bit, int end_bit, int32_t *hist, cudaStream_t st,
                       int32_t *launches) {
  if (n <= 1 || end_bit <= begin_bit) return cudaSuccess;
  const int32_t ntiles = (int32_t)((n + kSortTile - 1) / kSortTile);
  const int64_t nh = (int64_t)256 * ntiles;
  int32_t *counts = hist, *offs = hist + nh, *tiles = hist + 2 * nh;
  K *ka = keys, *kb = keys_tmp;
  int32_t *va = vals, *vb = vals_tmp;
  int passes = 0;
  for (int shift = begin_bit; shift < end_bit; shift += 8, ++passes) {
    k_sort_hist<K><<<ntiles, kSortNT, 0, st>>>(ka, n, shift, ntiles, counts);
    cudaError_t e = launch_xscan(counts, offs, nh, tiles, st);
    if (e != cudaSuccess) return e;
    k_sort_scatter<K><<<ntiles, kSortNT, 0, st>>>(ka, va, n, shift, ntiles, offs, kb, vb);
    std::swap(ka, kb);
    std::swap(va, vb);
    if (launches) *launches += 5;
  }
  if (passes & 1) {
    cudaError_t e = cudaMemcpyAsync(keys, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    if (vals) {
      e = cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

}  // namespace

// Sorts keys[0, n) (and vals alongside, if given) by bits [begin_bit,
// end_bit) of the keys, stably.  keys_tmp / vals_tmp: n entries each;
// hist: radix_sort_scratch_ints(n) ints.  The result ends in keys / vals.
// `launches` (optional) counts the kernels launched.
cudaError_t launch_radix_sort(unsigned long long *keys, unsigned long long *keys_tmp,
                              int32_t *vals, int32_t *vals_tmp, int64_t n, int begin_bit,
                              int end_bit, int32_t *hist, cudaStream_t st, int32_t *launches) {
  return radix_sort(keys, keys_tmp, vals, vals_tmp, n, begin_bit, end_bit, hist, st, launches);
}

cudaError_t launch_radix_sort(uint32_t *keys, uint32_t *keys_tmp, int32_t *vals,
                              int32_t *vals_tmp, int64_t n, int begin_bit, int end_bit,
                              int32_t *hist, cudaStream_t st, int32_t *launches) {
  return radix_sort(keys, keys_tmp, vals, vals_tmp, n, begin_bit, end_bit, hist, st, launches);
}

}  // namespace slg
