// Dense-core tile path: exact overlap counts of a dense 0/1 block on the
// fifth-generation tensor cores (tcgen05), the linear-algebra view of
// Section IV-D (B·Bᵀ) applied to the block only.
//
// A is an Mp x Kp matrix of bytes, 0x38 (E4M3 1.0) where a core row contains a
// core column and 0 elsewhere, row-major (K contiguous), Mp and Kp multiples
// of 128.  C = A·Aᵀ with FP32 accumulation is exact: every product is 0 or 1
// and every sum is at most Kp < 2^24, so the FP32 partial sums are integers
// represented exactly whatever the accumulation order.
//
// One CTA (4 warps) computes one 128 x 128 tile (bi, bj) with bj >= bi:
//   * thread 0 streams 128 x 128-byte slabs of rows bi and bj through a
//     two-stage shared-memory ring with TMA (cp.async.bulk.tensor, 128B
//     swizzle), and issues tcgen05.mma.kind::f8f6f4 (M = N = 128, K = 32 per
//     instruction) accumulating in 128 TMEM columns;
//   * all four warps read the accumulator back with tcgen05.ld (each warp its
//     32 TMEM lanes) and store it as int32.
// Every mbarrier wait is bounded; a wait that gives up sets an error flag and
// the CTA still releases its TMEM.
#include <cuda.h>

#include "slg_internal.cuh"

namespace slg {

namespace {

constexpr int kTcTile = 128;            // M = N tile
constexpr int kTcKBytes = 128;          // K slab per stage (one 128B swizzle row)
constexpr int kTcStages = 2;
constexpr int kTcSlab = kTcTile * kTcKBytes;  // 16 KB per operand per stage
constexpr uint32_t kTcCols = 128;       // TMEM columns (fp32 accumulator)
constexpr long kSpinLimit = 1L << 26;   // bounded waits

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with parity `parity` to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int32_t x,
                                            int32_t y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major operand, 128B swizzle,
// rows of 128 bytes, 8-row groups 1024 bytes apart.
//   [0,14) start address >> 4, [16,30) leading byte offset >> 4 (unused for
//   swizzled K-major; 1), [32,46) stride byte offset >> 4 (1024 B),
//   [46,48) version 1, [61,64) layout: 2 = 128B swizzle.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1u << 46;
  d |= (uint64_t)2u << 61;
  return d;
}

// Instruction descriptor, kind::f8f6f4: D = F32 (bits 4-5 = 1), A = B = E4M3
// (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bit 17,
// M >> 4 at bit 24.
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTcTile >> 3) << 17) |
                            ((uint32_t)(kTcTile >> 4) << 24);

__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

struct TcTask {
  int32_t bi, bj;
};

__global__ __launch_bounds__(128, 1) void k_tile_overlap(const __grid_constant__ CUtensorMap map,
                                                         int32_t Mp, int32_t Kp,
                                                         const TcTask *__restrict__ tasks,
                                                         int32_t *__restrict__ C,
                                                         int32_t *__restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the 128B-swizzled slabs
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char *sa = smem;                          // [stages][16 KB]
  unsigned char *sb = smem + kTcStages * kTcSlab;    // [stages][16 KB]
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + 2 * kTcStages * kTcSlab);
  uint64_t *empty = full + kTcStages;
  uint64_t *done = empty + kTcStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TcTask t = tasks[blockIdx.x];
  const int32_t nk = Kp / kTcKBytes;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTcCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (threadIdx.x == 0) {
    // prologue: fill the ring
    for (int s = 0; s < kTcStages && s < nk; ++s) {
      mbar_expect_tx(full + s, 2 * kTcSlab);
      tma_load_2d(sa + s * kTcSlab, &map, s * kTcKBytes, t.bi * kTcTile, full + s);
      tma_load_2d(sb + s * kTcSlab, &map, s * kTcKBytes, t.bj * kTcTile, full + s);
    }
    for (int32_t k = 0; k < nk && ok; ++k) {
      const int s = k % kTcStages;
      const uint32_t ph = (uint32_t)(k / kTcStages) & 1u;
      if (!mbar_wait(full + s, ph)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sa + s * kTcSlab), b0 = smem_u32(sb + s * kTcSlab);
#pragma unroll
      for (int kk = 0; kk < kTcKBytes / 32; ++kk) {
        // advance 32 bytes along K inside the swizzle row: +2 in address >> 4
        mma_f8(tmem, smem_desc_sw128(a0) + 2u * kk, smem_desc_sw128(b0) + 2u * kk,
               (k > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(empty + s);
      const int32_t kn = k + kTcStages;
      if (kn < nk) {
        // the slot is free once the MMAs that read it have completed
        if (!mbar_wait(empty + s, ph)) {
          ok = false;
          break;
        }
        mbar_expect_tx(full + s, 2 * kTcSlab);
        tma_load_2d(sa + s * kTcSlab, &map, kn * kTcKBytes, t.bi * kTcTile, full + s);
        tma_load_2d(sb + s * kTcSlab, &map, kn * kTcKBytes, t.bj * kTcTile, full + s);
      }
    }
    mma_commit(done);
    if (!ok) atomicExch(err, (int32_t)SLG_ERR_TIMEOUT);
  }
  __syncwarp();
  // everyone waits for the accumulator (bounded)
  if (!mbar_wait(done, 0)) atomicExch(err, (int32_t)SLG_ERR_TIMEOUT);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (*(volatile int32_t *)err == 0) {
    const int32_t row = t.bi * kTcTile + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < kTcTile; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
          "%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31},"
          " [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      int4 *dst = reinterpret_cast<int4 *>(C + (int64_t)row * Mp + t.bj * kTcTile + c0);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        dst[q] = make_int4((int32_t)__uint_as_float(v[4 * q + 0]),
                           (int32_t)__uint_as_float(v[4 * q + 1]),
                           (int32_t)__uint_as_float(v[4 * q + 2]),
                           (int32_t)__uint_as_float(v[4 * q + 3]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTcCols)
                 : "memory");
}

__global__ void k_tc_tasks(int32_t nt, TcTask *tasks) {
  // upper-triangle tile list: (bi, bj), bj >= bi
  const int32_t id = blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t total = nt * (nt + 1) / 2;
  if (id >= total) return;
  int32_t bi = 0, rem = id;
  while (rem >= nt - bi) {
    rem -= nt - bi;
    ++bi;
  }
  tasks[id] = TcTask{bi, bi + rem};
}

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    cudaGetLastError();
  }
  return fn;
}

}  // namespace

size_t tile_overlap_smem() { return 2 * kTcStages * kTcSlab + 1024 + 64; }

// C[Mp x Mp] (upper-triangle tiles written) = A·Aᵀ for A [Mp x Kp] bytes.
// `tasks` has room for nt (nt + 1) / 2 entries (nt = Mp / 128); `err` is a
// device int set to 1 if a bounded wait gave up.
cudaError_t launch_tile_overlap(const uint8_t *A, int32_t Mp, int32_t Kp, int32_t *C,
                                void *tasks, int32_t *err, cudaStream_t st) {
  if (Mp <= 0 || Kp <= 0 || Mp % kTcTile || Kp % kTcKBytes) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(A) & 15) != 0) return cudaErrorInvalidValue;
  EncodeTiled enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)Mp};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp};  // bytes between rows
  const cuuint32_t box[2] = {(cuuint32_t)kTcKBytes, (cuuint32_t)kTcTile};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(A), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const int32_t nt = Mp / kTcTile;
  const int32_t ntask = nt * (nt + 1) / 2;
  TcTask *tk = reinterpret_cast<TcTask *>(tasks);
  k_tc_tasks<<<(ntask + 255) / 256, 256, 0, st>>>(nt, tk);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tile_overlap, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tile_overlap_smem());
    attr = true;
  }
  k_tile_overlap<<<ntask, 128, tile_overlap_smem(), st>>>(map, Mp, Kp, tk, C, err);
  return cudaGetLastError();
}

}  // namespace slg
