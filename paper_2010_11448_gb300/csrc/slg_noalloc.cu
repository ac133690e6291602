// slg_count_noalloc: the pair count of L_s for callers that must not allocate
// device memory.  It runs a count-only variant of the plain per-hyperedge
// kernel whose working memory -- per-warp count arrays, per-warp bitmaps and
// a small result block -- lives in one fixed, file-scope device array instead
// of memory obtained from cudaMalloc or a pool.
//
// Host code never dereferences that array by name: in host code the symbol
// only stands in for the device array, so its device address is looked up
// with cudaGetSymbolAddress once per device (with that device current) and
// that address is what the kernels receive.
#include <mutex>

#include "slg_internal.cuh"

namespace slg {

namespace {

// 64 MiB of int32, zero at load; every GPU that loads the library keeps it
// until the process exits.
constexpr long long kNoallocInts = 16ll * 1024 * 1024;
constexpr int kNoallocResultInts = 128;  // Meta (error word, totals), 512 B, aligned
constexpr int kNoallocNT = 256;
constexpr int kNoallocMaxWarps = 1024;

static __device__ __align__(256) int32_t g_noalloc_scratch[kNoallocInts];

struct NoallocDevice {
  int32_t *base = nullptr;  // device address of g_noalloc_scratch
  bool ready = false;
  // Set when a call may have left non-zero counters or bitmap words behind
  // (it returned with an error after its memset).  A call that completes
  // sets every counter and bitmap word it touched back to zero, and the
  // array is zero when the library is loaded, so only then does the next
  // call clear more than the result block.
  bool dirty = false;
};

std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];

static_assert(sizeof(Meta) <= kNoallocResultInts * sizeof(int32_t), "result block too small");

// Count-only plain walk: one warp per hyperedge (cyclic), Algorithm 3's
// checks per wedge (f > e, |f| >= s), counts in the warp's dense array, one
// bit per 32 counters in the warp's bitmap; the pairs of each row with count
// >= s are added to meta->pairs, and the touched counters and bitmap words
// are set back to zero.
__global__ __launch_bounds__(kNoallocNT) void k_noalloc_count(Side sd, int32_t smin,
                                                              int32_t *__restrict__ counters,
                                                              uint32_t *__restrict__ bitmaps,
                                                              int32_t R_pad, int unweighted,
                                                              Meta *meta) {
  if (meta->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kNoallocNT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kNoallocNT) >> 5;
  const int32_t nsw = R_pad >> 10;
  int32_t *cnt = counters + gw * (int64_t)R_pad;
  uint32_t *sm = bitmaps + gw * (int64_t)nsw;
  unsigned long long pairs = 0;
  for (int64_t e = gw; e < sd.R; e += nw) {
    const int32_t lo = sd.r_off[e], hi = sd.r_off[e + 1];
    if (hi - lo < smin) continue;
    for (int32_t k = lo; k < hi; ++k) {
      const int32_t v = __ldg(sd.r_idx + k);
      const int32_t cb = __ldg(sd.c_off + v), ce = __ldg(sd.c_off + v + 1);
      for (int32_t q = cb + lane; q < ce; q += 32) {
        const int32_t f = __ldg(sd.c_idx + q);
        if (f <= e) continue;
        if (__ldg(sd.r_off + f + 1) - __ldg(sd.r_off + f) < smin) continue;
        if (unweighted && __ldcg(cnt + f) >= smin) continue;
        if (atomicAdd(cnt + f, 1) == 0) atomicOr(sm + (f >> 10), 1u << ((f >> 5) & 31));
      }
    }
    __threadfence_block();
    __syncwarp();
    for (int32_t w0 = 0; w0 < nsw; w0 += 32) {
      const int32_t sw = w0 + lane;
      if (sw >= nsw) continue;
      const uint32_t bits = __ldcg(sm + sw);
      for (uint32_t b = bits; b; b &= b - 1) {
        int4 *p = reinterpret_cast<int4 *>(cnt + ((sw << 10) | ((__ffs(b) - 1) << 5)));
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int4 x = __ldcg(p + q);
          pairs += (x.x >= smin) + (x.y >= smin) + (x.z >= smin) + (x.w >= smin);
          __stcg(p + q, make_int4(0, 0, 0, 0));
        }
      }
      if (bits) __stcg(sm + sw, 0u);
    }
    __threadfence_block();
    __syncwarp();
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, d);
  if (lane == 0 && pairs) atomicAdd(&meta->pairs, pairs);
}

// CSR and CSC must describe the same incidence: one warp per CSR row e
// looks e up in the (validated, ascending) column of each of its vertices.
// With nnz equal on both sides and strictly ascending rows and columns, a
// hit for every CSR incidence means the two are the same set.  Needs no
// memory beyond the inputs; a miss raises SLG_ERR_INVALID.
__global__ __launch_bounds__(kNoallocNT) void k_noalloc_agree(Side sd, Meta *meta) {
  if (meta->err) return;
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * kNoallocNT + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * kNoallocNT) >> 5;
  for (int64_t e = gw; e < sd.R; e += nw) {
    const int32_t lo = sd.r_off[e], hi = sd.r_off[e + 1];
    bool miss = false;
    for (int32_t k = lo + lane; k < hi; k += 32) {
      const int32_t v = __ldg(sd.r_idx + k);
      if (find_sorted(sd.c_idx, __ldg(sd.c_off + v), __ldg(sd.c_off + v + 1), (int32_t)e) < 0)
        miss = true;
    }
    if (__any_sync(0xffffffffu, miss) && lane == 0)
      raise_error(meta, SLG_ERR_INVALID, kWhereMismatch);
  }
}

// Device address of the static array for the current device (first call per
// device looks it up).
cudaError_t noalloc_base(int32_t **out, NoallocDevice **dv) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoallocDevice &d = g_noalloc_dev[dev % 64];
  *dv = &d;
  if (!d.ready) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    d.base = static_cast<int32_t *>(p);
    d.ready = true;
  }
  *out = d.base;
  return cudaSuccess;
}

}  // namespace

long long noalloc_warps_for(int32_t R) {
  const long long R_pad = ((long long)(R > 0 ? R : 1) + 1023) / 1024 * 1024;
  long long w = (kNoallocInts - kNoallocResultInts) / (R_pad + R_pad / 1024);
  w = (w / 8) * 8;
  return w > kNoallocMaxWarps ? kNoallocMaxWarps : w;
}

}  // namespace slg

using namespace slg;

extern "C" int slg_count_noalloc(const slg_hypergraph *h, int32_t s, uint32_t flags,
                                 int64_t *n_pairs, void *stream) {
  if (!h || !n_pairs || s < 1) return SLG_ERR_INVALID;
  if (h->n_edges < 0 || h->n_vertices < 0 || h->nnz < 0 || h->nnz >= (int64_t(1) << 31))
    return SLG_ERR_INVALID;
  if (!h->e_off || !h->v_off || (h->nnz > 0 && (!h->e_idx || !h->v_idx))) return SLG_ERR_INVALID;
  if (flags & ~(uint32_t)(SLG_DUAL | SLG_UNWEIGHTED)) return SLG_ERR_INVALID;
  Side sd;
  sd.nnz = h->nnz;
  const bool dual = (flags & SLG_DUAL) != 0;
  sd.R = dual ? h->n_vertices : h->n_edges;
  sd.C = dual ? h->n_edges : h->n_vertices;
  sd.r_off = dual ? h->v_off : h->e_off;
  sd.r_idx = dual ? h->v_idx : h->e_idx;
  sd.c_off = dual ? h->e_off : h->v_off;
  sd.c_idx = dual ? h->e_idx : h->v_idx;
  const long long warps = noalloc_warps_for(sd.R);
  if (warps < 8) return SLG_ERR_TOO_LARGE;
  const long long R_pad = ((long long)(sd.R > 0 ? sd.R : 1) + 1023) / 1024 * 1024;

  cudaStream_t st = (cudaStream_t)stream;
  int32_t *base = nullptr;
  NoallocDevice *dv = nullptr;
  cudaError_t e = noalloc_base(&base, &dv);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SLG_ERR_CUDA;
  }
  Meta *meta = reinterpret_cast<Meta *>(base);
  int32_t *counters = base + kNoallocResultInts;
  uint32_t *bitmaps = reinterpret_cast<uint32_t *>(counters + warps * R_pad);
  // What must start at zero: the result block always; the counters and
  // bitmaps this call uses only after a call that may have stopped early.
  bool clear_all;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    clear_all = dv->dirty;
    dv->dirty = true;  // until this call has finished cleanly
  }
  const size_t used = clear_all ? (size_t)(kNoallocResultInts + warps * R_pad +
                                           warps * (R_pad / 1024))
                                : (size_t)kNoallocResultInts;
  if (cudaMemsetAsync(base, 0, used * sizeof(int32_t), st) != cudaSuccess) {
    cudaGetLastError();
    return SLG_ERR_CUDA;
  }
  // Input checks on the device (offsets, id ranges, ascending rows, CSR and
  // CSC the same incidence) before the walk reads anything through them.
  if (launch_validate(sd, meta, st) != cudaSuccess) {
    cudaGetLastError();
    return SLG_ERR_CUDA;
  }
  const int grid = (int)((warps * 32 + kNoallocNT - 1) / kNoallocNT);
  k_noalloc_agree<<<grid, kNoallocNT, 0, st>>>(sd, meta);
  k_noalloc_count<<<grid, kNoallocNT, 0, st>>>(sd, s, counters, bitmaps, (int32_t)R_pad,
                                              (flags & SLG_UNWEIGHTED) ? 1 : 0, meta);
  if (cudaGetLastError() != cudaSuccess) return SLG_ERR_CUDA;
  Meta m;
  if (cudaMemcpyAsync(&m, meta, sizeof(Meta), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return SLG_ERR_CUDA;
  }
  if (!m.err) {
    // the count kernel ran to the end: every counter it touched is zero again
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    dv->dirty = false;
  }
  if (m.err) return m.err;
  *n_pairs = (int64_t)m.pairs;
  return SLG_OK;
}
