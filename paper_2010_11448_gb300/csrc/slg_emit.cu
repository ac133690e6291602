// Output assembly: the exclusive scan of the per-row pair counts gives every
// row its place in the canonical (i, j)-ordered edge list (rows in ascending
// i, each row's pairs already in ascending j), and the gather copies the
// staged rows there.  This replaces the paper's concatenation of thread-local
// edge vectors (Section IV-F) with a deterministic layout.
#include "slg_internal.cuh"

namespace slg {

namespace {

constexpr int kNT = 256;
constexpr int kIPT = 16;
constexpr int kTile = kNT * kIPT;

__global__ __launch_bounds__(kNT) void k_rowscan_reduce(const int32_t *__restrict__ n_e,
                                                        int32_t rows, long long *__restrict__ tile,
                                                        const Meta *meta) {
  if (meta->err) return;
  __shared__ long long ws[kNT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  long long c = 0;
  for (int i = 0; i < kIPT; ++i) {
    const int64_t r = base + (int64_t)i * kNT + threadIdx.x;
    if (r < rows) c += n_e[r];
  }
  long long total;
  block_inclusive_scan64<kNT>(c, ws, &total);
  if (threadIdx.x == 0) tile[blockIdx.x] = total;
}

__global__ __launch_bounds__(1024) void k_scan_tiles64(long long *tile, int32_t n, Meta *meta) {
  if (meta->err) return;
  __shared__ long long ws[1024 / 32 + 1];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int32_t base = 0; base < n; base += 1024) {
    const int32_t i = base + threadIdx.x;
    const long long x = i < n ? tile[i] : 0;
    long long total;
    const long long inc = block_inclusive_scan64<1024>(x, ws, &total);
    if (i < n) tile[i] = carry + inc - x;
    __syncthreads();
    if (threadIdx.x == 0) carry += total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    tile[n] = carry;
    meta->pairs = (unsigned long long)carry;
  }
}

__global__ __launch_bounds__(kNT) void k_rowscan_apply(const int32_t *__restrict__ n_e, int32_t rows,
                                                       const long long *__restrict__ tile,
                                                       long long *__restrict__ row_ptr,
                                                       int32_t ntiles, const Meta *meta) {
  if (meta->err) return;
  __shared__ long long ws[kNT / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * kTile;
  long long carry = tile[blockIdx.x];
  for (int i = 0; i < kIPT; ++i) {
    const int64_t r = base + (int64_t)i * kNT + threadIdx.x;
    const long long x = r < rows ? n_e[r] : 0;
    long long total;
    const long long inc = block_inclusive_scan64<kNT>(x, ws, &total);
    if (r < rows) row_ptr[r] = carry + inc - x;
    carry += total;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) row_ptr[rows] = tile[ntiles];
}

constexpr int kGatherRows = 256;
constexpr int kGatherQ = 4;  // positions per thread whose loads are in flight together

// A block owns kGatherRows consecutive rows and copies their staged pairs to
// the output range [row_ptr[r0], row_ptr[r0 + rows)), each thread finding its
// row by binary search over the block's offsets.
__global__ __launch_bounds__(kNT) void k_gather(int32_t row_begin, int32_t rows,
                                                const long long *__restrict__ row_ptr,
                                                const long long *__restrict__ stage_pos,
                                                const int32_t *__restrict__ stage_j,
                                                const int32_t *__restrict__ stage_w,
                                                int32_t *__restrict__ out_i,
                                                int32_t *__restrict__ out_j,
                                                int32_t *__restrict__ out_w, int unweighted,
                                                long long stage_cap, long long out_cap,
                                                Meta *meta) {
  if (meta->err) return;
  __shared__ long long s_ptr[kGatherRows + 1];
  __shared__ long long s_sp[kGatherRows];
  const int32_t r0 = blockIdx.x * kGatherRows;
  const int32_t nr = min(kGatherRows, rows - r0);
  for (int i = threadIdx.x; i <= nr; i += kNT) s_ptr[i] = row_ptr[r0 + i];
  for (int i = threadIdx.x; i < nr; i += kNT) s_sp[i] = stage_pos[r0 + i];
  __syncthreads();
  const long long p1 = s_ptr[nr];
  // A thread's positions ascend, so its row index only moves forward: the
  // next row is searched for only when p has left the current one, and the
  // loads of kGatherQ positions are issued before their stores.
  int lo = 0;  // s_ptr[lo] <= p for every p still to come
  for (long long p0 = s_ptr[0] + threadIdx.x; p0 < p1; p0 += (long long)kGatherQ * kNT) {
    long long src[kGatherQ];
    int row[kGatherQ];
#pragma unroll
    for (int q = 0; q < kGatherQ; ++q) {
      const long long p = p0 + (long long)q * kNT;
      src[q] = -1;
      row[q] = lo;
      if (p < p1) {
        if (s_ptr[lo + 1] <= p) {  // past the row: binary search in (lo, nr)
          int a = lo + 1, hi = nr;  // s_ptr[a] <= p < s_ptr[hi]
          while (hi - a > 1) {
            const int mid = (a + hi) >> 1;
            if (s_ptr[mid] <= p) a = mid;
            else hi = mid;
          }
          lo = a;
        }
        row[q] = lo;
        src[q] = s_sp[lo] < 0 ? -2 : s_sp[lo] + (p - s_ptr[lo]);
      }
    }
    int32_t vj[kGatherQ], vw[kGatherQ];
#pragma unroll
    for (int q = 0; q < kGatherQ; ++q) {
      const bool ok = src[q] >= 0 && src[q] < stage_cap;
      vj[q] = ok ? stage_j[src[q]] : 0;
      vw[q] = ok && !unweighted ? stage_w[src[q]] : 0;
    }
#pragma unroll
    for (int q = 0; q < kGatherQ; ++q) {
      const long long p = p0 + (long long)q * kNT;
      if (p >= p1) continue;
      if (src[q] < 0 || src[q] >= stage_cap || p >= out_cap) {  // more pairs than counted
        raise_error(meta, SLG_ERR_INVALID, kWhereStage);
        continue;
      }
      if (out_i) out_i[p] = row_begin + r0 + row[q];  // null: compressed row form
      out_j[p] = vj[q];
      if (!unweighted) out_w[p] = vw[q];
    }
  }
}

// w16[i] = w[i] for i < n, 8 weights per thread step (two 16-byte loads, one
// 16-byte store); a weight above 65,535 sets *bad.  Both arrays start on a
// 16-byte boundary (pool allocations).
__global__ __launch_bounds__(kNT) void k_pack_w16(const int32_t *__restrict__ w, long long n,
                                                  uint16_t *__restrict__ w16,
                                                  int32_t *__restrict__ bad) {
  const long long n8 = n >> 3;
  const long long stride = (long long)gridDim.x * kNT;
  bool over = false;
  for (long long q = (long long)blockIdx.x * kNT + threadIdx.x; q < n8; q += stride) {
    const int4 a = reinterpret_cast<const int4 *>(w)[2 * q];
    const int4 b = reinterpret_cast<const int4 *>(w)[2 * q + 1];
    over |= ((uint32_t)(a.x | a.y | a.z | a.w | b.x | b.y | b.z | b.w) > 0xFFFFu);
    uint4 o;
    o.x = (uint32_t)(a.x & 0xFFFF) | ((uint32_t)a.y << 16);
    o.y = (uint32_t)(a.z & 0xFFFF) | ((uint32_t)a.w << 16);
    o.z = (uint32_t)(b.x & 0xFFFF) | ((uint32_t)b.y << 16);
    o.w = (uint32_t)(b.z & 0xFFFF) | ((uint32_t)b.w << 16);
    reinterpret_cast<uint4 *>(w16)[q] = o;
  }
  for (long long i = (n8 << 3) + (long long)blockIdx.x * kNT + threadIdx.x; i < n; i += stride) {
    over |= ((uint32_t)w[i] > 0xFFFFu);
    w16[i] = (uint16_t)w[i];
  }
  if (over) *bad = 1;
}

__global__ void k_meta_copy(const uint32_t *__restrict__ src, volatile uint32_t *dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

}  // namespace

cudaError_t launch_pack_w16(const int32_t *w, int64_t n, uint16_t *w16, int32_t *bad,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long groups = (n + 7) / 8;
  const int blocks = (int)std::min<long long>((groups + kNT - 1) / kNT, 152 * 8);
  k_pack_w16<<<blocks, kNT, 0, st>>>(w, n, w16, bad);
  return cudaGetLastError();
}

cudaError_t launch_meta_copy(const Meta *src, Meta *dst, cudaStream_t st) {
  static_assert(sizeof(Meta) % 4 == 0, "Meta is copied as 32-bit words");
  k_meta_copy<<<1, 128, 0, st>>>(reinterpret_cast<const uint32_t *>(src),
                                 reinterpret_cast<volatile uint32_t *>(dst),
                                 (int)(sizeof(Meta) / 4));
  return cudaGetLastError();
}

cudaError_t launch_row_scan(int32_t rows, const Work &w, cudaStream_t st) {
  const int32_t ntiles = (rows + kTile - 1) / kTile;
  if (ntiles > 0) k_rowscan_reduce<<<ntiles, kNT, 0, st>>>(w.n_e, rows, w.tile64, w.meta);
  k_scan_tiles64<<<1, 1024, 0, st>>>(w.tile64, ntiles, w.meta);
  if (ntiles > 0)
    k_rowscan_apply<<<ntiles, kNT, 0, st>>>(w.n_e, rows, w.tile64, w.row_ptr, ntiles, w.meta);
  return cudaGetLastError();
}

cudaError_t launch_gather(int32_t row_begin, int32_t rows, const Work &w, int32_t *out_i,
                          int32_t *out_j, int32_t *out_w, int unweighted, long long out_cap,
                          cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const int grid = (rows + kGatherRows - 1) / kGatherRows;
  k_gather<<<grid, kNT, 0, st>>>(row_begin, rows, w.row_ptr, w.stage_pos, w.stage_j, w.stage_w,
                                 out_i, out_j, out_w, unweighted, w.stage_cap, out_cap, w.meta);
  return cudaGetLastError();
}

}  // namespace slg
