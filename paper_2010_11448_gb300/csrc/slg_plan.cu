// Batched form: many hypergraphs H_1 .. H_k, each with its own threshold s_g,
// computed as one hypergraph -- their disjoint union.  The union's incidence
// is block-diagonal (no vertex is shared between members), so every pair of
// the union's s-line graph lies inside one member, and with a per-row
// threshold (each row carries its member's s_g) the union's edge list is the
// concatenation of the members' edge lists, in member order, with ids
// shifted by the member's offsets.  One pipeline (one set of launches,
// capturable into a CUDA graph) serves the whole batch.
#include "slg_internal.cuh"

namespace slg {

namespace {

constexpr int kNT = 256;

// grid.y = member; blocks stride over the member's arrays.
__global__ __launch_bounds__(kNT) void k_concat(const BatchGraph *__restrict__ gs,
                                                int32_t *__restrict__ e_off,
                                                int32_t *__restrict__ e_idx,
                                                int32_t *__restrict__ v_off,
                                                int32_t *__restrict__ v_idx,
                                                int32_t *__restrict__ row_s_e,
                                                int32_t *__restrict__ row_s_v,
                                                int32_t *__restrict__ row_fhi_e,
                                                int32_t *__restrict__ row_fhi_v) {
  const BatchGraph g = gs[blockIdx.y];
  const int64_t t0 = (int64_t)blockIdx.x * kNT + threadIdx.x;
  const int64_t step = (int64_t)gridDim.x * kNT;
  for (int64_t i = t0; i < g.m; i += step) {
    e_off[g.e_base + i] = (int32_t)(g.e_off[i] + g.k_base);
    row_s_e[g.e_base + i] = g.s;
    row_fhi_e[g.e_base + i] = g.e_base + g.m;  // far ends stay inside the member
  }
  for (int64_t i = t0; i < g.n; i += step) {
    v_off[g.v_base + i] = (int32_t)(g.v_off[i] + g.k_base);
    row_s_v[g.v_base + i] = g.s;
    row_fhi_v[g.v_base + i] = g.v_base + g.n;
  }
  for (int64_t k = t0; k < g.nnz; k += step) {
    e_idx[g.k_base + k] = g.e_idx[k] + g.v_base;
    v_idx[g.k_base + k] = g.v_idx[k] + g.e_base;
  }
}

// Union ids -> member ids; offsets[g] = first pair of member g.
__global__ __launch_bounds__(kNT) void k_localize(int32_t *__restrict__ out_i,
                                                  int32_t *__restrict__ out_j, long long pairs,
                                                  const int32_t *__restrict__ row_base,
                                                  int32_t count,
                                                  const long long *__restrict__ row_ptr,
                                                  long long *__restrict__ offsets) {
  const long long t0 = (long long)blockIdx.x * kNT + threadIdx.x;
  const long long step = (long long)gridDim.x * kNT;
  if (t0 <= count) offsets[t0] = row_ptr[row_base[t0]];
  for (long long p = t0; p < pairs; p += step) {
    const int32_t i = out_i[p];
    int32_t a = 0, b = count;  // largest g with row_base[g] <= i
    while (b - a > 1) {
      const int32_t mid = (a + b) >> 1;
      if (__ldg(row_base + mid) <= i) a = mid;
      else b = mid;
    }
    const int32_t base = __ldg(row_base + a);
    out_i[p] = i - base;
    out_j[p] -= base;
  }
}

}  // namespace

cudaError_t launch_concat(const BatchGraph *g, int32_t count, int32_t max_len, int32_t *e_off,
                          int32_t *e_idx, int32_t *v_off, int32_t *v_idx, int32_t *row_s_e,
                          int32_t *row_s_v, int32_t *row_fhi_e, int32_t *row_fhi_v,
                          cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int gx = (max_len + kNT - 1) / kNT;
  if (gx < 1) gx = 1;
  if (gx > 1024) gx = 1024;
  dim3 grid(gx, count);
  k_concat<<<grid, kNT, 0, st>>>(g, e_off, e_idx, v_off, v_idx, row_s_e, row_s_v, row_fhi_e,
                                 row_fhi_v);
  return cudaGetLastError();
}

cudaError_t launch_localize(int32_t *out_i, int32_t *out_j, long long pairs,
                            const int32_t *row_base, int32_t count, const long long *row_ptr,
                            long long *offsets, cudaStream_t st) {
  long long g = (pairs + kNT - 1) / kNT;
  if (g < (count + kNT) / kNT) g = (count + kNT) / kNT;
  if (g > 65536) g = 65536;
  if (g < 1) g = 1;
  k_localize<<<(int)g, kNT, 0, st>>>(out_i, out_j, pairs, row_base, count, row_ptr, offsets);
  return cudaGetLastError();
}

}  // namespace slg
