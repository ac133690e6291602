// After the edge list: ID squeezing (Section IV-E), the line graph's
// adjacency, and s-connected components (the components of L_s, the
// motivating analysis of Section I).
//
// Squeezing numbers the ids that occur in the list 0 .. n_ids-1 in
// ascending order of their original id, so a canonical list stays
// canonical.  The adjacency is the symmetric CSR of L_s: row v lists its
// smaller neighbours (from a stable regrouping of the pairs by j) and then
// its larger ones (its own segment of the canonical list), both ascending.
// Components are found by lock-free union-find over the pairs: each root
// links to the smaller root, so every label ends as the smallest id of its
// component.
#include "slg_internal.cuh"

namespace slg {

namespace {

constexpr int kNT = 256;

int grid_for(int64_t items) {
  int64_t g = (items + kNT - 1) / kNT;
  if (g > 65536) g = 65536;
  return g < 1 ? 1 : (int)g;
}

// mark[v] = 1 for every id of the list (flags, int32 so that a scan counts).
__global__ __launch_bounds__(kNT) void k_mark(const int32_t *__restrict__ a,
                                              const int32_t *__restrict__ b, int64_t n,
                                              int32_t *__restrict__ mark) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += step) {
    mark[a[p]] = 1;
    mark[b[p]] = 1;
  }
}

// new id of v = rank[v] (exclusive scan of mark); old_of_new[rank[v]] = v.
__global__ __launch_bounds__(kNT) void k_squeeze_map(const int32_t *__restrict__ mark,
                                                     const int32_t *__restrict__ rank, int32_t R,
                                                     int32_t *__restrict__ old_of_new) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t v = (int64_t)blockIdx.x * kNT + threadIdx.x; v < R; v += step)
    if (mark[v]) old_of_new[rank[v]] = (int32_t)v;
}

__global__ __launch_bounds__(kNT) void k_squeeze_ids(const int32_t *__restrict__ a,
                                                     const int32_t *__restrict__ b, int64_t n,
                                                     const int32_t *__restrict__ rank,
                                                     int32_t *__restrict__ oa,
                                                     int32_t *__restrict__ ob) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += step) {
    oa[p] = __ldg(rank + a[p]);
    ob[p] = __ldg(rank + b[p]);
  }
}

// Degrees: up[i] += 1 and lo[j] += 1 per pair (i < j).
__global__ __launch_bounds__(kNT) void k_degrees(const int32_t *__restrict__ a,
                                                 const int32_t *__restrict__ b, int64_t n,
                                                 int32_t *__restrict__ up,
                                                 int32_t *__restrict__ lo) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += step) {
    atomicAdd(up + a[p], 1);
    atomicAdd(lo + b[p], 1);
  }
}

// deg[v] = lo[v] + up[v] as int64 scan input.
__global__ __launch_bounds__(kNT) void k_deg_sum(const int32_t *__restrict__ up,
                                                 const int32_t *__restrict__ lo, int32_t V,
                                                 long long *__restrict__ deg) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t v = (int64_t)blockIdx.x * kNT + threadIdx.x; v < V; v += step)
    deg[v] = (long long)up[v] + lo[v];
}

__global__ __launch_bounds__(1024) void k_scan64_inplace(long long *x, int64_t n) {
  __shared__ long long ws[1024 / 32 + 1];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b = 0; b < n; b += 1024) {
    const int64_t i = b + threadIdx.x;
    const long long v = i < n ? x[i] : 0;
    long long total;
    const long long inc = block_inclusive_scan64<1024>(v, ws, &total);
    if (i < n) x[i] = carry + inc - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) x[n] = carry;
}

// Upper neighbours: pair p of row i sits at p - first[i] within i's segment
// of the canonical list, first[i] = p of the segment's first pair.
__global__ __launch_bounds__(kNT) void k_seg_first(const int32_t *__restrict__ a, int64_t n,
                                                   long long *__restrict__ first) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += step)
    if (p == 0 || a[p - 1] != a[p]) first[a[p]] = p;
}

__global__ __launch_bounds__(kNT) void k_fill_upper(
    const int32_t *__restrict__ a, const int32_t *__restrict__ b, const int32_t *__restrict__ w,
    int64_t n, const long long *__restrict__ off, const int32_t *__restrict__ lo,
    const long long *__restrict__ first, int32_t *__restrict__ adj, int32_t *__restrict__ adj_w) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += step) {
    const int32_t i = a[p];
    const long long q = off[i] + lo[i] + (p - first[i]);
    adj[q] = b[p];
    if (adj_w) adj_w[q] = w[p];
  }
}

// Start of each group of the pairs regrouped by j.
__global__ __launch_bounds__(kNT) void k_group_first(const uint32_t *__restrict__ keys, int64_t n,
                                                     long long *__restrict__ lfirst) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t q = (int64_t)blockIdx.x * kNT + threadIdx.x; q < n; q += step)
    if (q == 0 || keys[q - 1] != keys[q]) lfirst[keys[q]] = q;
}

// Lower neighbours: element q of the stable regrouping by j (value = list
// position p) is the (q - lfirst[j])-th smaller neighbour of j, ascending
// because the canonical list meets j's pairs in ascending i.
__global__ __launch_bounds__(kNT) void k_fill_lower(
    const uint32_t *__restrict__ keys, const int32_t *__restrict__ pos,
    const int32_t *__restrict__ a, const int32_t *__restrict__ w, int64_t n,
    const long long *__restrict__ off, const long long *__restrict__ lfirst,
    int32_t *__restrict__ adj, int32_t *__restrict__ adj_w) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t q = (int64_t)blockIdx.x * kNT + threadIdx.x; q < n; q += step) {
    const int32_t j = (int32_t)keys[q];
    const long long dst = off[j] + (q - lfirst[j]);
    const int32_t p = pos[q];
    adj[dst] = a[p];
    if (adj_w) adj_w[dst] = w[p];
  }
}

// err = 1 if an id is outside [0, R) or i >= j; with `canonical`, also if
// the pairs are not strictly ascending in (i, j).
__global__ __launch_bounds__(kNT) void k_check_pairs(const int32_t *__restrict__ a,
                                                     const int32_t *__restrict__ b, int64_t n,
                                                     int32_t R, int canonical, int32_t *err) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += step) {
    const int32_t i = a[p], j = b[p];
    bool bad = i < 0 || j < 0 || i >= R || j >= R || i >= j;
    if (canonical && p > 0) {
      const int32_t pi = a[p - 1], pj = b[p - 1];
      bad |= pi > i || (pi == i && pj >= j);
    }
    if (bad) atomicExch(err, 1);
  }
}

__global__ __launch_bounds__(kNT) void k_iota(int32_t *__restrict__ x, int64_t n) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t v = (int64_t)blockIdx.x * kNT + threadIdx.x; v < n; v += step) x[v] = (int32_t)v;
}

__global__ __launch_bounds__(kNT) void k_keys_u32(const int32_t *__restrict__ b, int64_t n,
                                                  uint32_t *__restrict__ keys) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += step)
    keys[p] = (uint32_t)b[p];
}

constexpr int kMaxUnionSteps = 1 << 25;  // above any path length (ids < 2^24): a guard

__device__ __forceinline__ int32_t find_root(int32_t *parent, int32_t v) {
  // path halving; parents only decrease, so the walk ends at a root
  for (int step = 0; step < kMaxUnionSteps; ++step) {
    const int32_t p = parent[v];
    if (p == v) return v;
    const int32_t gp = parent[p];
    if (gp != p) atomicMin(parent + v, gp);
    v = gp;
  }
  return -1;
}

__global__ __launch_bounds__(kNT) void k_union(const int32_t *__restrict__ a,
                                               const int32_t *__restrict__ b, int64_t n,
                                               int32_t *__restrict__ parent, int32_t *err) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t p = (int64_t)blockIdx.x * kNT + threadIdx.x; p < n; p += step) {
    int32_t x = a[p], y = b[p];
    int tries = 0;
    for (; tries < kMaxUnionSteps; ++tries) {
      x = find_root(parent, x);
      y = find_root(parent, y);
      if (x < 0 || y < 0) break;
      if (x == y) break;
      if (x > y) {
        const int32_t t = x;
        x = y;
        y = t;
      }
      // link the larger root under the smaller one; fails if y stopped
      // being a root meanwhile, then retry from the new roots
      if (atomicCAS(parent + y, y, x) == y) break;
    }
    if (tries >= kMaxUnionSteps || x < 0 || y < 0) atomicExch(err, 1);
  }
}

__global__ __launch_bounds__(kNT) void k_flatten(int32_t *__restrict__ parent, int32_t R,
                                                 const int32_t *__restrict__ mark,
                                                 unsigned long long *__restrict__ n_comp,
                                                 int32_t *err) {
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t v = (int64_t)blockIdx.x * kNT + threadIdx.x; v < R; v += step) {
    const int32_t r = find_root(parent, (int32_t)v);
    if (r < 0) {
      atomicExch(err, 1);
      continue;
    }
    parent[v] = r;
    if (r == v && mark[v]) atomicAdd(n_comp, 1ull);
  }
}

}  // namespace

cudaError_t launch_mark(const int32_t *a, const int32_t *b, int64_t n, int32_t *mark,
                        cudaStream_t st) {
  if (n > 0) k_mark<<<grid_for(n), kNT, 0, st>>>(a, b, n, mark);
  return cudaGetLastError();
}

cudaError_t launch_squeeze(const int32_t *a, const int32_t *b, int64_t n, int32_t R,
                           const int32_t *mark, const int32_t *rank, int32_t *oa, int32_t *ob,
                           int32_t *old_of_new, cudaStream_t st) {
  if (R > 0) k_squeeze_map<<<grid_for(R), kNT, 0, st>>>(mark, rank, R, old_of_new);
  if (n > 0) k_squeeze_ids<<<grid_for(n), kNT, 0, st>>>(a, b, n, rank, oa, ob);
  return cudaGetLastError();
}

// deg scratch: up, lo [V] (zeroed by the caller); off [V + 1].
cudaError_t launch_adjacency_offsets(const int32_t *a, const int32_t *b, int64_t n, int32_t V,
                                     int32_t *up, int32_t *lo, long long *off,
                                     cudaStream_t st) {
  if (n > 0) k_degrees<<<grid_for(n), kNT, 0, st>>>(a, b, n, up, lo);
  if (V > 0) k_deg_sum<<<grid_for(V), kNT, 0, st>>>(up, lo, V, off);
  k_scan64_inplace<<<1, 1024, 0, st>>>(off, V);
  return cudaGetLastError();
}

cudaError_t launch_check_pairs(const int32_t *a, const int32_t *b, int64_t n, int32_t R,
                               int canonical, int32_t *err, cudaStream_t st) {
  if (n > 0) k_check_pairs<<<grid_for(n), kNT, 0, st>>>(a, b, n, R, canonical, err);
  return cudaGetLastError();
}

// first, lfirst [V] int64 scratch; keys, keys_tmp (u32), pos, pos_tmp [n];
// hist radix_sort_scratch_ints(n).
cudaError_t launch_adjacency_fill(const int32_t *a, const int32_t *b, const int32_t *w,
                                  int64_t n, int32_t V, const long long *off, const int32_t *lo,
                                  long long *first, long long *lfirst, uint32_t *keys,
                                  uint32_t *keys_tmp, int32_t *pos, int32_t *pos_tmp,
                                  int32_t *hist, int32_t *adj, int32_t *adj_w, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_seg_first<<<grid_for(n), kNT, 0, st>>>(a, n, first);
  k_fill_upper<<<grid_for(n), kNT, 0, st>>>(a, b, w, n, off, lo, first, adj, adj_w);
  k_keys_u32<<<grid_for(n), kNT, 0, st>>>(b, n, keys);
  k_iota<<<grid_for(n), kNT, 0, st>>>(pos, n);
  int bits = 0;
  while (bits < 31 && ((int64_t)(V > 0 ? V - 1 : 0) >> bits) != 0) ++bits;
  cudaError_t e = launch_radix_sort(keys, keys_tmp, pos, pos_tmp, n, 0, bits, hist, st);
  if (e != cudaSuccess) return e;
  k_group_first<<<grid_for(n), kNT, 0, st>>>(keys, n, lfirst);
  k_fill_lower<<<grid_for(n), kNT, 0, st>>>(keys, pos, a, w, n, off, lfirst, adj, adj_w);
  return cudaGetLastError();
}

cudaError_t launch_components(const int32_t *a, const int32_t *b, int64_t n, int32_t R,
                              int32_t *labels, const int32_t *mark, unsigned long long *n_comp,
                              int32_t *err, cudaStream_t st) {
  if (R > 0) k_iota<<<grid_for(R), kNT, 0, st>>>(labels, R);
  if (n > 0) k_union<<<grid_for(n), kNT, 0, st>>>(a, b, n, labels, err);
  if (R > 0) k_flatten<<<grid_for(R), kNT, 0, st>>>(labels, R, mark, n_comp, err);
  return cudaGetLastError();
}

}  // namespace slg
