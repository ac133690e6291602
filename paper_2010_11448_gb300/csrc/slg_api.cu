// C ABI of the slg library (declared in include/slg.h): argument checks,
// per-call working memory, the sequence of planning, walking and output
// kernels, and the single device->host read of the pair count.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "slg_internal.cuh"

namespace slg {
namespace {

constexpr int kMaxDevices = 64;

// Per-device state kept between calls: the plain kernel's dense counters
// (all zero between calls; the kernel restores the zeros it disturbs).
struct DeviceCtx {
  std::mutex mu;               // the plain kernel's scratch
  int32_t *giant = nullptr;    // plain kernel: per-warp zeroed counters
  size_t giant_elems = 0;
  std::mutex mem_mu;           // creation of `mem`
  cudaMemPool_t mem = nullptr;  // the library's stream-ordered memory pool
};

DeviceCtx g_ctx[kMaxDevices];

DeviceCtx &ctx_for_current(int *dev_out) {
  int dev = 0;
  cudaGetDevice(&dev);
  *dev_out = dev;
  return g_ctx[dev % kMaxDevices];
}

// The library's own stream-ordered memory pool on the current device,
// created on first use.  Freed memory stays in it for the next call (release
// threshold unlimited), and memory freed on one stream is reused on another
// only once the free has completed: the pool never makes a call wait for
// another stream's work, so calls on different streams overlap (e.g. one
// build's copies to the host with the next build's walk).  Null if the pool
// cannot be created (the device's default pool is used then).
cudaMemPool_t lib_pool() {
  int dev = 0;
  DeviceCtx &c = ctx_for_current(&dev);
  std::lock_guard<std::mutex> lock(c.mem_mu);
  if (!c.mem) {
    cudaMemPoolProps p = {};
    p.allocType = cudaMemAllocationTypePinned;
    p.handleTypes = cudaMemHandleTypeNone;
    p.location.type = cudaMemLocationTypeDevice;
    p.location.id = dev;
    if (cudaMemPoolCreate(&c.mem, &p) == cudaSuccess) {
      uint64_t thr = ~0ull;
      cudaMemPoolSetAttribute(c.mem, cudaMemPoolAttrReleaseThreshold, &thr);
      int off = 0;
      cudaMemPoolSetAttribute(c.mem, cudaMemPoolReuseAllowInternalDependencies, &off);
    } else {
      c.mem = nullptr;
    }
    cudaGetLastError();
  }
  return c.mem;
}
thread_local slg_stats t_stats;
thread_local int t_profile = 0;
thread_local int32_t t_tau_c = 64, t_tau_r = 32;
thread_local Bins t_bins;
thread_local float t_min_density = 0.02f;

// Validation and the CSR->CSC maps of both sides of one device input, made
// once for several builds on it (slg_build_host_many, slg_graph_*).  While
// t_prep points to one, run() on the same input skips its own validation and
// map.
struct Prepared {
  slg_hypergraph h{};
  int32_t *map[2] = {nullptr, nullptr};  // side H, side H*
};
thread_local const Prepared *t_prep = nullptr;

bool same_input(const slg_hypergraph &a, const slg_hypergraph &b) {
  return a.n_edges == b.n_edges && a.n_vertices == b.n_vertices && a.nnz == b.nnz &&
         a.e_off == b.e_off && a.e_idx == b.e_idx && a.v_off == b.v_off && a.v_idx == b.v_idx;
}

// t_prep for the lifetime of a scope
struct PrepScope {
  explicit PrepScope(const Prepared *p) { t_prep = p; }
  ~PrepScope() { t_prep = nullptr; }
};

// Events of one profiled call: plan start, walk (kNumBins + 1), scan end,
// gather start and end, relabel start and end, re-ordering start and end.
struct Events {
  cudaEvent_t ev[kNumBins + 11] = {};
  bool on = false;
  explicit Events(bool enable) {
    if (!enable) return;
    for (auto &e : ev)
      if (cudaEventCreate(&e) != cudaSuccess) return;
    on = true;
  }
  ~Events() {
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
  }
  float ms(int a, int b) const {
    float t = 0.f;
    if (on && cudaEventElapsedTime(&t, ev[a], ev[b]) != cudaSuccess) {
      cudaGetLastError();
      t = 0.f;
    }
    return t;
  }
};
// Event slots.
constexpr int kEvPlan = 0, kEvWalk = 1, kEvScan = kNumBins + 2, kEvGather0 = kNumBins + 3,
              kEvGather1 = kNumBins + 4, kEvRelabel0 = kNumBins + 5, kEvRelabel1 = kNumBins + 6,
              kEvOrder0 = kNumBins + 7, kEvOrder1 = kNumBins + 8, kEvTile0 = kNumBins + 9,
              kEvTile1 = kNumBins + 10;

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return SLG_OK;
  if (e == cudaErrorMemoryAllocation) return SLG_ERR_NOMEM;
  return SLG_ERR_CUDA;
}

// When an allocation fails, the pool's unused memory goes back to the
// driver and the allocation is tried once more, so that memory the pool
// keeps never starves an allocation (the pool's own, or a plain cudaMalloc).
void trim_pool() {
  cudaMemPool_t m = lib_pool();
  if (m) cudaMemPoolTrimTo(m, 0);
  cudaGetLastError();
}

// Stream-ordered allocations released (stream-ordered) when the call ends.
struct Pool {
  cudaStream_t st;
  cudaMemPool_t mem;
  std::vector<void *> ptrs;
  explicit Pool(cudaStream_t s) : st(s), mem(lib_pool()) {}
  cudaError_t alloc(void **q, size_t bytes) {
    return mem ? cudaMallocFromPoolAsync(q, bytes, mem, st) : cudaMallocAsync(q, bytes, st);
  }
  template <class T>
  cudaError_t get(T **p, size_t count) {
    size_t bytes = count * sizeof(T);
    if (bytes < 16) bytes = 16;
    void *q = nullptr;
    cudaError_t e = alloc(&q, bytes);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      cudaStreamSynchronize(st);  // frees queued on the stream complete first
      trim_pool();
      e = alloc(&q, bytes);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return e;
    }
    ptrs.push_back(q);
    *p = static_cast<T *>(q);
    return cudaSuccess;
  }
  ~Pool() {
    for (void *q : ptrs) cudaFreeAsync(q, st);
  }
};

// With the environment variable SLG_DEBUG set, every failing CUDA step is
// reported on stderr with its source expression (host side only).
bool debug_on() {
  static const bool on = std::getenv("SLG_DEBUG") != nullptr;
  return on;
}

cudaError_t debug_fail(cudaError_t e, const char *what, int line) {
  if (e != cudaSuccess && debug_on())
    std::fprintf(stderr, "slg: line %d: %s: %s\n", line, what, cudaGetErrorString(e));
  return e;
}

#define SLG_TRY(expr)                                          \
  do {                                                         \
    cudaError_t _e = debug_fail((expr), #expr, __LINE__);      \
    if (_e != cudaSuccess) {                                   \
      cudaGetLastError();                                      \
      return status_of(_e);                                    \
    }                                                          \
  } while (0)

int check_args(const slg_hypergraph *h, int32_t s, uint32_t flags) {
  if (!h || s < 1) return SLG_ERR_INVALID;
  if (h->n_edges < 0 || h->n_vertices < 0 || h->nnz < 0 || h->nnz >= (int64_t(1) << 31))
    return SLG_ERR_INVALID;
  if (!h->e_off || !h->v_off) return SLG_ERR_INVALID;
  if (h->nnz > 0 && (!h->e_idx || !h->v_idx)) return SLG_ERR_INVALID;
  const uint32_t algo = flags & SLG_ALGO_MASK;
  if (algo != SLG_ALGO_BINNED && algo != SLG_ALGO_PLAIN && algo != SLG_ALGO_SPGEMM)
    return SLG_ERR_UNSUPPORTED;
  if (flags & ~(uint32_t)(SLG_DUAL | SLG_UNWEIGHTED | SLG_TENSOR_CORE | SLG_RELABEL_ASC |
                          SLG_RELABEL_DESC | SLG_NO_PRUNE | SLG_ALGO_MASK))
    return SLG_ERR_INVALID;
  if ((flags & SLG_NO_PRUNE) && algo != SLG_ALGO_BINNED) return SLG_ERR_UNSUPPORTED;
  if ((flags & SLG_RELABEL_ASC) && (flags & SLG_RELABEL_DESC)) return SLG_ERR_INVALID;
  if ((flags & SLG_TENSOR_CORE) && algo != SLG_ALGO_BINNED) return SLG_ERR_UNSUPPORTED;
  return SLG_OK;
}

Side side_of(const slg_hypergraph *h, uint32_t flags) {
  Side s;
  s.nnz = h->nnz;
  if (flags & SLG_DUAL) {
    s.R = h->n_vertices;
    s.C = h->n_edges;
    s.r_off = h->v_off;
    s.r_idx = h->v_idx;
    s.c_off = h->e_off;
    s.c_idx = h->e_idx;
  } else {
    s.R = h->n_edges;
    s.C = h->n_vertices;
    s.r_off = h->e_off;
    s.r_idx = h->e_idx;
    s.c_off = h->v_off;
    s.c_idx = h->v_idx;
  }
  return s;
}


cudaError_t ensure_giant(DeviceCtx &c, size_t elems, cudaStream_t st) {
  if (c.giant_elems >= elems) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  if (c.giant) cudaFree(c.giant);
  c.giant = nullptr;
  c.giant_elems = 0;
  e = cudaMalloc(&c.giant, elems * sizeof(int32_t));
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    trim_pool();
    e = cudaMalloc(&c.giant, elems * sizeof(int32_t));
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    c.giant = nullptr;
    return e;
  }
  e = cudaMemset(c.giant, 0, elems * sizeof(int32_t));
  if (e != cudaSuccess) return e;
  c.giant_elems = elems;
  return cudaSuccess;
}

enum Op { kOpCount, kOpBuild, kOpWedges };

// Everything one call needs after argument checks.
struct Call {
  Side sd;
  int32_t smin;
  uint32_t flags;
  bool unweighted;
  int32_t row_begin, row_end, rows;
  int32_t R_pad;
  Op op;
  int32_t *out_i, *out_j, *out_w;
  int32_t *row_work_out;  // slg_row_work: per-row wedge work (device)
  bool tile_ran;          // the dense-core tile kernel was launched
  int64_t capacity;
  cudaStream_t st;
  DeviceCtx *ctx;
  Pool *pool;
  Work w;
  Events *evs;
  int32_t launches;
  int64_t core_rows, core_cols, core_nnz;
  Meta *meta_host;  // this host thread's pinned copy of the device Meta
  Meta *meta_view;  // the same memory as the device addresses it
};

// One pinned Meta per host thread (calls on different threads and streams
// run concurrently; each reads its own results).
// This host thread's copy of the device Meta: pinned and mapped, so that a
// kernel writes it (read_meta) without the copy engines, which may be busy
// with large copies of other work (the results of slg_build_host_many).
cudaError_t thread_meta(Meta **out, Meta **view = nullptr) {
  thread_local Meta *m = nullptr, *v = nullptr;
  if (!m) {
    cudaError_t e = cudaHostAlloc(&m, sizeof(Meta), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&v), m, 0);
    if (e != cudaSuccess) {
      if (m) cudaFreeHost(m);
      m = v = nullptr;
      return e;
    }
  }
  *out = m;
  if (view) *view = v;
  return cudaSuccess;
}

int plain_warps() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 4;  // 4 warps per SM: a multiple of 8 (the kernel's block)
}

// Zero-initialised scratch of the plain kernel: per-warp dense counters
// followed by the per-warp bitmaps (kept zero between calls).
cudaError_t ensure_scratch(Call &c, size_t *summ_off) {
  const size_t pw = (size_t)plain_warps();
  const size_t rp = (size_t)c.R_pad;
  const size_t counters = pw * rp;
  *summ_off = counters;
  return ensure_giant(*c.ctx, counters + pw * (rp >> 10), c.st);
}

// Per-CTA scratch of the giant bin: 4 ints per wedge of the largest row.
cudaError_t giant_scratch(Call &c, int32_t max_work, WalkLaunch *L) {
  L->giant_scratch = nullptr;
  L->giant_stride = 0;
  if (max_work <= 0) return cudaSuccess;
  const long long stride = 4ll * max_work;
  cudaError_t e = c.pool->get(&L->giant_scratch, (size_t)giant_ctas() * (size_t)stride);
  if (e == cudaSuccess) L->giant_stride = stride;
  return e;
}

thread_local int32_t t_err_where = 0;  // kWhere* of the last device-raised error

int read_meta(Call &c) {
  SLG_TRY(launch_meta_copy(c.w.meta, c.meta_view, c.st));
  SLG_TRY(cudaStreamSynchronize(c.st));
  if (c.meta_host->err) t_err_where = c.meta_host->err_where;
  return c.meta_host->err;
}

WalkLaunch walk_launch(Call &c, int mode, int32_t smin, int32_t list_base) {
  WalkLaunch L = {};
  L.a.mode = mode;
  L.a.unweighted = c.unweighted;
  L.a.row_s = c.sd.row_s;
  L.a.row_fhi = c.sd.row_fhi;
  L.a.dense_ratio = t_bins.dense;
  L.a.smin = smin;
  L.a.row_begin = list_base;
  L.a.n_e = c.w.n_e;
  L.a.stage_pos = c.w.stage_pos;
  L.a.stage_j = c.w.stage_j;
  L.a.stage_w = c.w.stage_w;
  L.a.stage_cap = c.w.stage_cap;
  L.a.meta = c.w.meta;
  L.a.row_work = c.w.row_work;
  L.bin_rows = c.w.bin_rows;
  L.row_work = c.w.row_work;
  L.rows = c.rows;
  L.R = c.sd.R;
  return L;
}

// Dense core for SLG_TENSOR_CORE: core flags and ranks, a host decision on
// the block's size and density, the core-excluded column lists, packing and
// the tensor-core tile counts.  Leaves `core` zero when no block qualifies.
int plan_core(Call &c, CoreInfo *core) {
  *core = CoreInfo{};
  Work &w = c.w;
  const Side &sd = c.sd;
  int32_t *core_col, *col_rank, *core_row, *row_rank, *tile;
  SLG_TRY(c.pool->get(&core_col, (size_t)sd.C + 1));
  SLG_TRY(c.pool->get(&col_rank, (size_t)sd.C + 1));
  SLG_TRY(c.pool->get(&core_row, (size_t)sd.R + 1));
  SLG_TRY(c.pool->get(&row_rank, (size_t)sd.R + 1));
  const int64_t nt = std::max(xscan_tiles((int64_t)sd.C + 1), xscan_tiles((int64_t)sd.R + 1));
  SLG_TRY(c.pool->get(&tile, (size_t)nt + 1));
  SLG_TRY(launch_core_cols(sd, t_tau_c, core_col, w.meta, c.st));
  SLG_TRY(launch_xscan(core_col, col_rank, (int64_t)sd.C + 1, tile, c.st));
  SLG_TRY(launch_core_rows(sd, t_tau_r, col_rank, core_row, &w.meta->nnz_core, w.meta, c.st));
  SLG_TRY(launch_xscan(core_row, row_rank, (int64_t)sd.R + 1, tile, c.st));
  c.launches += 8;
  int32_t sizes[2] = {0, 0};
  SLG_TRY(cudaMemcpyAsync(&sizes[0], row_rank + sd.R, 4, cudaMemcpyDeviceToHost, c.st));
  int rc = read_meta(c);
  if (rc) return rc;
  if (sizes[0] < 128) return SLG_OK;
  // Refinement: the core columns are the columns where the core rows
  // concentrate (at least max(8, min_density x |core rows|) of them); then the
  // core rows are taken again against those columns.  This drops high-degree
  // columns that the core rows hardly use.
  {
    int32_t *col_cnt;
    SLG_TRY(c.pool->get(&col_cnt, (size_t)sd.C + 1));
    const int32_t tau2 = std::max<int32_t>(8, (int32_t)std::ceil(t_min_density * sizes[0]));
    SLG_TRY(launch_core_refine(sd, row_rank, col_cnt, tau2, core_col, w.meta, c.st));
    SLG_TRY(launch_xscan(core_col, col_rank, (int64_t)sd.C + 1, tile, c.st));
    SLG_TRY(cudaMemsetAsync(&w.meta->nnz_core, 0, sizeof(unsigned long long), c.st));
    SLG_TRY(launch_core_rows(sd, t_tau_r, col_rank, core_row, &w.meta->nnz_core, w.meta, c.st));
    SLG_TRY(launch_xscan(core_row, row_rank, (int64_t)sd.R + 1, tile, c.st));
    c.launches += 7;
  }
  SLG_TRY(cudaMemcpyAsync(&sizes[0], row_rank + sd.R, 4, cudaMemcpyDeviceToHost, c.st));
  SLG_TRY(cudaMemcpyAsync(&sizes[1], col_rank + sd.C, 4, cudaMemcpyDeviceToHost, c.st));
  rc = read_meta(c);
  if (rc) return rc;
  const int64_t nR = sizes[0], nC = sizes[1];
  const int64_t nnz_core = (int64_t)c.meta_host->nnz_core;
  const int32_t kept = c.meta_host->kept;
  if (nR < 128 || nC < 32 || (double)nnz_core < (double)t_min_density * (double)nR * (double)nC)
    return SLG_OK;
  const int64_t Mp = (nR + 127) / 128 * 128, Kp = (nC + 127) / 128 * 128;
  if (Mp * Kp > (int64_t(1) << 31) || Mp * Mp > (int64_t(1) << 30) || Kp >= (1 << 24))
    return SLG_OK;  // block too large for the tile path: plain walk
  int32_t *core_list, *x_cnt, *x_off, *T;
  uint8_t *A;
  SLG_TRY(c.pool->get(&core_list, (size_t)nR));
  SLG_TRY(c.pool->get(&x_cnt, (size_t)nC + 1));
  SLG_TRY(c.pool->get(&x_off, (size_t)nC + 1));
  SLG_TRY(launch_core_list(sd.R, row_rank, core_list, c.st));
  SLG_TRY(cudaMemsetAsync(x_cnt, 0, sizeof(int32_t) * (nC + 1), c.st));
  SLG_TRY(launch_core_xcount(sd.C, col_rank, w.c_off_s, w.c_idx_s, row_rank, x_cnt, w.meta,
                             c.st));
  SLG_TRY(launch_xscan(x_cnt, x_off, nC + 1, tile, c.st));
  // the core-excluded lists go right after the kept entries (c_idx_s has
  // room for 2 x nnz entries when the flag is set; they are at most nnz)
  SLG_TRY(launch_core_xcsc(sd.C, col_rank, w.c_off_s, w.c_idx_s, row_rank, x_off,
                           w.c_idx_s + kept, w.meta, c.st));
  SLG_TRY(c.pool->get(&A, (size_t)(Mp * Kp)));
  SLG_TRY(c.pool->get(&T, (size_t)(Mp * Mp)));
  void *tasks = nullptr;
  const int64_t ntile = Mp / 128;
  SLG_TRY(c.pool->get(reinterpret_cast<int64_t **>(&tasks), (size_t)(ntile * (ntile + 1) / 2)));
  SLG_TRY(cudaMemsetAsync(A, 0, (size_t)(Mp * Kp), c.st));
  SLG_TRY(launch_core_pack(sd, row_rank, col_rank, A, (int32_t)Kp, w.meta, c.st));
  if (c.evs->on) cudaEventRecord(c.evs->ev[kEvTile0], c.st);
  cudaError_t e = launch_tile_overlap(A, (int32_t)Mp, (int32_t)Kp, T, tasks, &w.meta->err, c.st);
  if (c.evs->on) cudaEventRecord(c.evs->ev[kEvTile1], c.st);
  if (e == cudaErrorNotSupported) return SLG_ERR_UNSUPPORTED;
  SLG_TRY(e);
  c.launches += 7;
  c.tile_ran = true;
  core->row_rank = row_rank;
  core->col_rank = col_rank;
  core->x_off = x_off;
  core->x_base = kept;
  core->core_list = core_list;
  core->n_core = (int32_t)nR;
  core->T = T;
  core->Mp = (int32_t)Mp;
  c.core_rows = nR;
  c.core_cols = nC;
  c.core_nnz = nnz_core;
  return SLG_OK;
}

// Default path: filtered CSC, binned single walk, staging, scan, gather.
int run_binned(Call &c, int64_t *result) {
  Work &w = c.w;
  // Degree-based pruning (Alg. 3) drops rows of size < s from both ends of
  // the walk; SLG_NO_PRUNE keeps them (the threshold still applies to the
  // counts, and such rows cannot reach it).
  const int32_t s_prune = (c.flags & SLG_NO_PRUNE) ? 1 : c.smin;
  SLG_TRY(launch_filter(c.sd, s_prune, w, c.st));
  CoreInfo core = {};
  if (c.flags & SLG_TENSOR_CORE) {
    const int rcc = plan_core(c, &core);
    if (rcc) return rcc;
  }
  SLG_TRY(launch_rows_work(c.sd, s_prune, c.row_begin, c.row_end, w, core, t_bins, c.st));
  c.launches += 4 + (c.rows > 0 ? 1 : 0);
  if (c.op == kOpWedges) {
    if (c.row_work_out)
      SLG_TRY(cudaMemcpyAsync(c.row_work_out, w.row_work, sizeof(int32_t) * (size_t)c.rows,
                              cudaMemcpyDeviceToDevice, c.st));
    int rc = read_meta(c);
    if (rc) return rc;
    *result = (int64_t)c.meta_host->wedges;
    return SLG_OK;
  }
  if (c.op == kOpBuild && c.capacity > 0) {
    if (c.pool->get(&w.stage_j, (size_t)c.capacity) == cudaSuccess &&
        (c.unweighted || c.pool->get(&w.stage_w, (size_t)c.capacity) == cudaSuccess))
      w.stage_cap = c.capacity;
    else
      w.stage_cap = 0;  // rows that find no staging room are re-walked directly
  }
  // Planning totals: the giant bin's scratch is sized by its largest row.
  int rc = read_meta(c);
  if (rc) return rc;
  // (core rows may have no wedges but still need a giant CTA; their pairs,
  // staged in the same scratch, also come from up to n_core tile items)
  // (a sparse-bin row whose candidates overflow its table is handed to the
  // giant bin, so the giant scratch also covers the sparse rows)
  const Meta &mp = *c.meta_host;
  const int32_t max_giant =
      (mp.rows_bin[kBinGiant] || mp.rows_bin[kBinSparse])
          ? std::max(std::max(mp.max_giant_work, mp.max_sparse_work), (int32_t)1) +
                (core.T ? core.n_core : 0)
          : 0;
  // the giant bin's list as planned (the walk may append overflow rows)
  const unsigned long long giant_rows0 = mp.rows_bin[kBinGiant];
  const unsigned giant_rest0 = mp.giant_rest;
  WalkLaunch L = walk_launch(c, c.op == kOpBuild ? kStage : kCount, c.smin, c.row_begin);
  L.a.core = core;
  SLG_TRY(giant_scratch(c, max_giant, &L));
  L.w.r_off = c.sd.r_off;
  L.w.r_idx = c.sd.r_idx;
  L.w.c_idx_s = w.c_idx_s;
  L.w.tail_beg = w.tail_beg;
  L.w.tail_end = w.tail_end;
  cudaEvent_t *ev = c.evs->on ? c.evs->ev + kEvWalk : nullptr;
  if (c.rows > 0) {
    SLG_TRY(launch_walk(L, c.st, &c.launches, ev));
  } else if (ev) {
    for (int b = 0; b <= kNumBins; ++b) cudaEventRecord(ev[b], c.st);
  }
  SLG_TRY(launch_row_scan(c.rows, w, c.st));
  if (c.evs->on) cudaEventRecord(c.evs->ev[kEvScan], c.st);
  c.launches += 3;
  rc = read_meta(c);
  if (rc) return rc;
  const Meta &m = *c.meta_host;
  const int64_t pairs = (int64_t)m.pairs;
  *result = pairs;
  if (c.op != kOpBuild) return SLG_OK;
  if (pairs > c.capacity) return SLG_ERR_CAPACITY;
  if (c.evs->on) cudaEventRecord(c.evs->ev[kEvGather0], c.st);
  if (pairs > 0) {
    if (m.stage_overflow == 0) {
      SLG_TRY(launch_gather(c.row_begin, c.rows, w, c.out_i, c.out_j, c.out_w, c.unweighted,
                            c.capacity, c.st));
      c.launches += 1;
    } else {
      // Staging too small: walk again, writing straight to the output.
      SLG_TRY(cudaMemsetAsync(&w.meta->giant_ticket, 0, sizeof(unsigned int), c.st));
      static_assert(offsetof(Meta, sparse_ticket_rest) ==
                        offsetof(Meta, sparse_ticket) + sizeof(unsigned int),
                    "the two sparse ticket counters are cleared together");
      SLG_TRY(cudaMemsetAsync(&w.meta->sparse_ticket, 0, 2 * sizeof(unsigned int), c.st));
      // back to the planned giant list: the sparse bin hands the same rows
      // over again
      SLG_TRY(cudaMemcpyAsync(&w.meta->rows_bin[kBinGiant], &giant_rows0, sizeof(giant_rows0),
                              cudaMemcpyHostToDevice, c.st));
      SLG_TRY(cudaMemcpyAsync(&w.meta->giant_rest, &giant_rest0, sizeof(giant_rest0),
                              cudaMemcpyHostToDevice, c.st));
      L.a.mode = kDirect;
      L.a.row_ptr = w.row_ptr;
      L.a.out_i = c.out_i;
      L.a.out_j = c.out_j;
      L.a.out_w = c.out_w;
      SLG_TRY(launch_walk(L, c.st, &c.launches));
    }
  }
  if (c.evs->on) cudaEventRecord(c.evs->ev[kEvGather1], c.st);
  rc = read_meta(c);
  return rc;
}

// Plain comparison path: count pass, scan, write pass (two walks).  Its
// per-warp count arrays are a persistent zeroed scratch shared by the
// device's calls, so plain calls are serialised per device.
int run_plain(Call &c, int64_t *result) {
  std::lock_guard<std::mutex> lock(c.ctx->mu);
  Work &w = c.w;
  size_t summ_off = 0;
  SLG_TRY(ensure_scratch(c, &summ_off));
  const int32_t pw = plain_warps();
  EmitArgs a = {};
  a.mode = kCount;
  a.unweighted = c.unweighted;
  a.smin = c.smin;
  a.row_begin = c.row_begin;
  a.n_e = w.n_e;
  a.meta = w.meta;
  uint32_t *summ = reinterpret_cast<uint32_t *>(c.ctx->giant + summ_off);
  if (c.evs->on) cudaEventRecord(c.evs->ev[kEvWalk], c.st);
  if (c.rows > 0)
    SLG_TRY(launch_plain(c.sd, c.smin, c.row_begin, c.row_end, a, c.ctx->giant, summ, c.R_pad,
                         pw, c.st));
  if (c.evs->on)
    for (int b = 1; b <= kNumBins; ++b) cudaEventRecord(c.evs->ev[kEvWalk + b], c.st);
  SLG_TRY(launch_row_scan(c.rows, w, c.st));
  if (c.evs->on) cudaEventRecord(c.evs->ev[kEvScan], c.st);
  c.launches += 4;
  int rc = read_meta(c);
  if (rc) return rc;
  const int64_t pairs = (int64_t)c.meta_host->pairs;
  *result = c.op == kOpWedges ? (int64_t)c.meta_host->wedges : pairs;
  if (c.op != kOpBuild) return SLG_OK;
  if (pairs > c.capacity) return SLG_ERR_CAPACITY;
  if (c.evs->on) cudaEventRecord(c.evs->ev[kEvGather0], c.st);
  if (pairs > 0 && c.rows > 0) {
    a.mode = kDirect;
    a.row_ptr = w.row_ptr;
    a.out_i = c.out_i;
    a.out_j = c.out_j;
    a.out_w = c.out_w;
    SLG_TRY(launch_plain(c.sd, c.smin, c.row_begin, c.row_end, a, c.ctx->giant, summ, c.R_pad,
                         pw, c.st));
    c.launches += 1;
  }
  if (c.evs->on) cudaEventRecord(c.evs->ev[kEvGather1], c.st);
  return read_meta(c);
}

// Filtered SpGEMM comparison path: product rows (full columns, both
// triangles, threshold 1) materialised chunk by chunk, then filtered.
int run_spgemm(Call &c, int64_t *result) {
  Work &w = c.w;
  const int32_t rows = c.rows;
  int32_t *work = nullptr, *kept = nullptr;
  long long *prefix = nullptr, *chunk_ptr = nullptr;
  SLG_TRY(c.pool->get(&work, (size_t)rows + 1));
  SLG_TRY(c.pool->get(&kept, (size_t)rows + 1));
  SLG_TRY(c.pool->get(&prefix, (size_t)rows + 1));
  SLG_TRY(c.pool->get(&chunk_ptr, (size_t)rows + 1));
  // 1. product-row sizes (upper bounds: sum of column lengths) and prefix
  SLG_TRY(launch_rows_full(c.sd, c.row_begin, c.row_end, c.row_begin, w.tail_beg, w.tail_end,
                           work, w.n_e, w.stage_pos, nullptr, rows, w.meta, c.st));
  Work wp = w;
  wp.n_e = work;
  wp.row_ptr = prefix;
  SLG_TRY(launch_row_scan(rows, wp, c.st));
  c.launches += 4;
  std::vector<long long> pre((size_t)rows + 1);
  SLG_TRY(cudaMemcpyAsync(pre.data(), prefix, sizeof(long long) * (rows + 1),
                          cudaMemcpyDeviceToHost, c.st));
  int rc = read_meta(c);
  if (rc) return rc;
  const long long total_work = pre[rows];
  if (c.op == kOpWedges) {
    *result = total_work;
    return SLG_OK;
  }
  // 2. staging budget for one chunk of product rows
  long long budget = total_work < (1ll << 30) ? total_work : (1ll << 30);
  long long max_row = 0;
  for (int32_t r = 0; r < rows; ++r)
    if (pre[r + 1] - pre[r] > max_row) max_row = pre[r + 1] - pre[r];
  if (budget < max_row) budget = max_row;
  if (budget < 1) budget = 1;
  SLG_TRY(c.pool->get(&w.stage_j, (size_t)budget));
  SLG_TRY(c.pool->get(&w.stage_w, (size_t)budget));
  w.stage_cap = budget;
  WalkLaunch Lg = walk_launch(c, kStage, 1, c.row_begin);
  Lg.a.full_rows = 1;
  SLG_TRY(giant_scratch(c, max_row > kCtaLMaxWork ? (int32_t)max_row : 0, &Lg));
  long long total_out = 0, products = 0;
  int32_t r0 = 0;
  if (c.evs->on) cudaEventRecord(c.evs->ev[kEvWalk], c.st);
  while (r0 < rows) {
    int32_t r1 = r0 + 1;
    while (r1 < rows && pre[r1 + 1] - pre[r0] <= budget) ++r1;
    const int32_t a0 = c.row_begin + r0, a1 = c.row_begin + r1;
    SLG_TRY(cudaMemsetAsync(w.meta, 0, sizeof(Meta), c.st));
    SLG_TRY(launch_rows_full(c.sd, a0, a1, c.row_begin, w.tail_beg, w.tail_end, w.row_work,
                             w.n_e, w.stage_pos, w.bin_rows, rows, w.meta, c.st));
    WalkLaunch L = Lg;
    L.w.r_off = c.sd.r_off;
    L.w.r_idx = c.sd.r_idx;
    L.w.c_idx_s = c.sd.c_idx;
    L.w.tail_beg = w.tail_beg;
    L.w.tail_end = w.tail_end;
    SLG_TRY(launch_walk(L, c.st, &c.launches));
    SLG_TRY(launch_filter_count(a0, a1, c.row_begin, w, c.smin, kept, c.st));
    Work wf = w;
    wf.n_e = kept;
    wf.row_ptr = chunk_ptr;
    SLG_TRY(launch_row_scan(r1 - r0, wf, c.st));
    c.launches += 5;
    rc = read_meta(c);
    if (rc) return rc;
    const Meta &m = *c.meta_host;
    if (m.stage_overflow) return SLG_ERR_NOMEM;  // cannot happen: chunk fits the budget
    const long long got = (long long)m.pairs;
    products += (long long)m.stage_cursor;
    if (c.op == kOpBuild && total_out + got <= c.capacity && got > 0) {
      SLG_TRY(launch_filter_write(a0, a1, c.row_begin, w, c.smin, chunk_ptr, total_out,
                                  c.unweighted, c.out_i, c.out_j, c.out_w, c.st));
      c.launches += 1;
    }
    total_out += got;
    r0 = r1;
  }
  if (c.evs->on) {
    for (int b = 1; b <= kNumBins; ++b) cudaEventRecord(c.evs->ev[kEvWalk + b], c.st);
    cudaEventRecord(c.evs->ev[kEvScan], c.st);
    cudaEventRecord(c.evs->ev[kEvGather0], c.st);
    cudaEventRecord(c.evs->ev[kEvGather1], c.st);
  }
  rc = read_meta(c);
  if (rc) return rc;
  c.meta_host->pairs = (unsigned long long)total_out;
  c.meta_host->wedges = (unsigned long long)total_work;
  c.meta_host->stage_cursor = (unsigned long long)products;
  *result = total_out;
  if (c.op == kOpBuild && total_out > c.capacity) return SLG_ERR_CAPACITY;
  return SLG_OK;
}

// The whole pipeline for one side, one s and one row range.
int run(const slg_hypergraph *h, int32_t smin, uint32_t flags, int32_t row_begin,
        int32_t row_end, Op op, int32_t *out_i, int32_t *out_j, int32_t *out_w,
        int64_t capacity, int64_t *result, cudaStream_t st, const int32_t *row_s = nullptr,
        int32_t *max_row_work = nullptr, long long *row_ptr_out = nullptr,
        int32_t *row_work_out = nullptr, const int32_t *row_fhi = nullptr) {
  int rc = check_args(h, smin, flags);
  if (rc != SLG_OK) return rc;
  if (!result) return SLG_ERR_INVALID;
  Call c = {};
  c.sd = side_of(h, flags);
  c.sd.row_s = row_s;
  c.sd.row_fhi = row_fhi;
  if (row_begin < 0 || row_end < row_begin || row_end > c.sd.R) return SLG_ERR_INVALID;
  c.smin = smin;
  c.flags = flags;
  c.unweighted = (flags & SLG_UNWEIGHTED) != 0;
  // Compressed row form (a build with row_ptr_out): the pairs' i is implied
  // by row_ptr_out, so out_i may be null.
  const bool rows_form = op == kOpBuild && row_ptr_out != nullptr;
  if (op == kOpBuild) {
    if (capacity < 0) return SLG_ERR_INVALID;
    if (capacity > 0 && ((!rows_form && !out_i) || !out_j || (!c.unweighted && !out_w)))
      return SLG_ERR_INVALID;
  }
  if (rows_form && ((flags & SLG_ALGO_MASK) == SLG_ALGO_SPGEMM ||
                    (flags & (SLG_RELABEL_ASC | SLG_RELABEL_DESC))))
    return SLG_ERR_UNSUPPORTED;
  c.row_begin = row_begin;
  c.row_end = row_end;
  c.rows = row_end - row_begin;
  c.op = op;
  c.out_i = out_i;
  c.out_j = out_j;
  c.out_w = out_w;
  c.capacity = capacity;
  c.st = st;
  c.row_work_out = row_work_out;
  const int64_t nnz = c.sd.nnz;
  c.R_pad = (int32_t)(((int64_t)c.sd.R + 1023) / 1024 * 1024);
  if (c.R_pad == 0) c.R_pad = 1024;
  if (c.sd.R > kMaxRows) return SLG_ERR_UNSUPPORTED;
  const uint32_t relabel = flags & (SLG_RELABEL_ASC | SLG_RELABEL_DESC);
  if (relabel && (row_begin != 0 || row_end != c.sd.R || row_s)) return SLG_ERR_UNSUPPORTED;

  int dev = 0;
  DeviceCtx &ctx = ctx_for_current(&dev);
  SLG_TRY(thread_meta(&c.meta_host, &c.meta_view));
  c.ctx = &ctx;

  Events evs(t_profile != 0 && op != kOpWedges);
  Pool pool(st);
  c.pool = &pool;
  c.evs = &evs;
  Work &w = c.w;
  const int32_t ntiles = (int32_t)((nnz + 4095) / 4096);
  const int32_t ntiles64 = (c.rows + 4095) / 4096;
  // a prepared input (validated, maps made): its map of this side is used
  // as it is (read only; relabelling makes its own)
  const Prepared *pp = (t_prep && !relabel && same_input(t_prep->h, *h)) ? t_prep : nullptr;
  SLG_TRY(pool.get(&w.meta, 1));
  if (pp) w.csr2csc = pp->map[(flags & SLG_DUAL) ? 1 : 0];
  else SLG_TRY(pool.get(&w.csr2csc, (size_t)nnz));
  SLG_TRY(pool.get(&w.qs, (size_t)nnz + 1));
  SLG_TRY(pool.get(&w.c_idx_s, (size_t)nnz * ((flags & SLG_TENSOR_CORE) ? 2 : 1) + 1));
  SLG_TRY(pool.get(&w.c_off_s, (size_t)c.sd.C + 1));
  SLG_TRY(pool.get(&w.tail_beg, (size_t)nnz));
  SLG_TRY(pool.get(&w.tail_end, (size_t)nnz));
  SLG_TRY(pool.get(&w.tile, (size_t)ntiles + 1));
  SLG_TRY(pool.get(&w.bin_rows, (size_t)kNumBins * (c.rows > 0 ? c.rows : 1)));
  SLG_TRY(pool.get(&w.n_e, (size_t)c.rows + 1));
  SLG_TRY(pool.get(&w.row_work, (size_t)c.rows + 1));
  SLG_TRY(pool.get(&w.stage_pos, (size_t)c.rows + 1));
  SLG_TRY(pool.get(&w.row_ptr, (size_t)c.rows + 1));
  SLG_TRY(pool.get(&w.tile64, (size_t)ntiles64 + 1));
  SLG_TRY(cudaMemsetAsync(w.meta, 0, sizeof(Meta), st));

  // Validation and the CSR->CSC map (a consistency check for every path),
  // unless the input was prepared.
  if (evs.on) cudaEventRecord(evs.ev[kEvPlan], st);
  if (!pp) {
    SLG_TRY(launch_validate(c.sd, w.meta, st));
    SLG_TRY(launch_csr2csc(c.sd, w.csr2csc, w.meta, st));
    c.launches += 3;
  }

  // Degree-ordered relabelling: the rest of the call runs on a renumbered
  // copy of the side (built only from input that passed validation).
  int32_t *perm = nullptr;
  if (relabel) {
    rc = read_meta(c);
    if (rc) return rc;
    int32_t *r_off2, *r_idx2, *c_idx2, *scr;
    SLG_TRY(pool.get(&perm, (size_t)c.sd.R + 1));
    SLG_TRY(pool.get(&r_off2, (size_t)c.sd.R + 1));
    SLG_TRY(pool.get(&r_idx2, (size_t)nnz + 1));
    SLG_TRY(pool.get(&c_idx2, (size_t)nnz + 1));
    SLG_TRY(pool.get(&scr, relabel_scratch_ints(c.sd.R, nnz)));
    if (evs.on) cudaEventRecord(evs.ev[kEvRelabel0], st);
    SLG_TRY(launch_relabel(c.sd, relabel == SLG_RELABEL_DESC, perm, r_off2, r_idx2, c_idx2, scr,
                           st, &c.launches));
    c.sd.r_off = r_off2;
    c.sd.r_idx = r_idx2;
    c.sd.c_idx = c_idx2;
    SLG_TRY(launch_csr2csc(c.sd, w.csr2csc, w.meta, st));
    if (evs.on) cudaEventRecord(evs.ev[kEvRelabel1], st);
    c.launches += 1;
  }

  int64_t value = 0;
  const uint32_t algo = flags & SLG_ALGO_MASK;
  if (algo == SLG_ALGO_PLAIN) rc = run_plain(c, &value);
  else if (algo == SLG_ALGO_SPGEMM) rc = run_spgemm(c, &value);
  else rc = run_binned(c, &value);
  if (rc == SLG_OK || rc == SLG_ERR_CAPACITY) *result = value;
  if (rc != SLG_OK) return rc;
  if (row_ptr_out) {
    SLG_TRY(cudaMemcpyAsync(row_ptr_out, w.row_ptr, sizeof(long long) * ((size_t)c.rows + 1),
                            cudaMemcpyDeviceToDevice, st));
    SLG_TRY(cudaStreamSynchronize(st));
  }

  // Relabelled pairs -> caller ids in canonical (i, j) order.
  if (perm && op == kOpBuild && value > 0) {
    if (value >= ((int64_t)1 << 31)) return SLG_ERR_UNSUPPORTED;
    unsigned long long *keys;
    int32_t *vals = nullptr, *hist;
    SLG_TRY(pool.get(&keys, 2 * (size_t)value));
    if (!c.unweighted) SLG_TRY(pool.get(&vals, (size_t)value));
    SLG_TRY(pool.get(&hist, radix_sort_scratch_ints(value)));
    if (evs.on) cudaEventRecord(evs.ev[kEvOrder0], st);
    SLG_TRY(launch_unrelabel(value, c.sd.R, perm, out_i, out_j, c.unweighted ? nullptr : out_w,
                             keys, vals, hist, st, &c.launches));
    if (evs.on) cudaEventRecord(evs.ev[kEvOrder1], st);
    SLG_TRY(cudaStreamSynchronize(st));
  }

  slg_stats stats = {};
  const Meta &m = *c.meta_host;
  stats.wedges = (int64_t)m.wedges;
  stats.pairs = op == kOpWedges ? 0 : value;
  stats.rows_active = (int64_t)m.active;
  for (int b = 0; b < kNumBins; ++b) {
    stats.rows_bin[b] = (int64_t)m.rows_bin[b];
    stats.wedges_bin[b] = (int64_t)m.wedges_bin[b];
    stats.incid_bin[b] = (int64_t)m.incid_bin[b];
    stats.pairs_bin[b] = (int64_t)m.pairs_bin[b];
  }
  if (max_row_work) *max_row_work = m.max_row_work;
  stats.kernel_launches = c.launches;
  stats.core_rows = c.core_rows;
  stats.core_cols = c.core_cols;
  stats.core_nnz = c.core_nnz;
  for (int q = 0; q < 4; ++q) stats.giant_cycles[q] = (int64_t)m.giant_cycles[q];
  for (int q = 0; q < 5; ++q) stats.sparse_cycles[q] = (int64_t)m.sparse_cycles[q];
  stats.max_row_work = m.max_row_work;
  if (evs.on) {
    stats.profiled = 1;
    stats.ms_plan = evs.ms(kEvPlan, kEvWalk);
    for (int b = 0; b < kNumBins; ++b)
      stats.ms_walk[b] = evs.ms(kEvWalk + kWalkEv[b], kEvWalk + kWalkEv[b] + 1);
    stats.ms_scan = evs.ms(kEvWalk + kNumBins, kEvScan);
    if (op == kOpBuild) stats.ms_gather = evs.ms(kEvGather0, kEvGather1);
    if (c.tile_ran) stats.ms_tile = evs.ms(kEvTile0, kEvTile1);
    if (perm) {
      stats.ms_relabel = evs.ms(kEvRelabel0, kEvRelabel1);
      if (op == kOpBuild && value > 0) stats.ms_order = evs.ms(kEvOrder0, kEvOrder1);
    }
  }
  t_stats = stats;
  return SLG_OK;
}


// ------------------------------------------------------------ batched form --

// Device memory owned by a plan (released by slg_plan_destroy).
struct Owned {
  std::vector<void *> ptrs;
  template <class T>
  cudaError_t get(T **p, size_t count) {
    size_t bytes = count * sizeof(T);
    if (bytes < 16) bytes = 16;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e == cudaErrorMemoryAllocation) {
      cudaGetLastError();
      trim_pool();
      e = cudaMalloc(&q, bytes);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return e;
    }
    ptrs.push_back(q);
    *p = static_cast<T *>(q);
    return cudaSuccess;
  }
  ~Owned() {
    for (void *q : ptrs) cudaFree(q);
  }
};

}  // namespace
}  // namespace slg

struct slg_plan {
  int dev = 0;
  uint32_t flags = 0;
  int32_t count = 0;
  slg_hypergraph u = {};           // the union (device arrays owned below)
  slg::Side sd = {};
  int32_t *row_s_e = nullptr, *row_s_v = nullptr;
  int32_t *row_fhi_e = nullptr, *row_fhi_v = nullptr;  // end of each row's member
  int32_t *row_base = nullptr;     // [count + 1] first row of each member (side)
  slg::Work w = {};
  int32_t *giant = nullptr;
  long long giant_stride = 0;
  int32_t *out_i = nullptr, *out_j = nullptr, *out_w = nullptr;
  long long *offsets = nullptr;    // [count + 1]
  int64_t pairs = 0;
  slg::Bins bins;
  float tuned_ms = 0.f;
  int32_t launches = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  slg::Owned mem;
};

namespace slg {
namespace {

// The whole build of a plan, enqueued without any host synchronisation.
#define PLAN_TRY(expr)                                          \
  do {                                                          \
    const cudaError_t _e = debug_fail((expr), #expr, __LINE__); \
    if (_e != cudaSuccess) return _e;                           \
  } while (0)

cudaError_t enqueue_plan(slg_plan *p, const Bins &bins, cudaStream_t st, int32_t *launches) {
  Work &w = p->w;
  const Side &sd = p->sd;
  PLAN_TRY(cudaMemsetAsync(w.meta, 0, sizeof(Meta), st));
  PLAN_TRY(launch_validate(sd, w.meta, st));
  PLAN_TRY(launch_csr2csc(sd, w.csr2csc, w.meta, st));
  PLAN_TRY(launch_filter(sd, 1, w, st));
  PLAN_TRY(launch_rows_work(sd, 1, 0, sd.R, w, CoreInfo{}, bins, st));
  WalkLaunch L = {};
  L.w.r_off = sd.r_off;
  L.w.r_idx = sd.r_idx;
  L.w.c_idx_s = w.c_idx_s;
  L.w.tail_beg = w.tail_beg;
  L.w.tail_end = w.tail_end;
  L.a.mode = kStage;
  L.a.unweighted = (p->flags & SLG_UNWEIGHTED) != 0;
  L.a.row_s = sd.row_s;
  L.a.row_fhi = sd.row_fhi;
  L.a.dense_ratio = bins.dense;
  L.a.smin = 1;
  L.a.row_begin = 0;
  L.a.n_e = w.n_e;
  L.a.stage_pos = w.stage_pos;
  L.a.stage_j = w.stage_j;
  L.a.stage_w = w.stage_w;
  L.a.stage_cap = w.stage_cap;
  L.a.meta = w.meta;
  L.a.row_work = w.row_work;
  L.bin_rows = w.bin_rows;
  L.row_work = w.row_work;
  L.rows = sd.R;
  L.R = sd.R;
  L.giant_scratch = p->giant;
  L.giant_stride = p->giant_stride;
  int32_t n = 0;
  if (sd.R > 0) PLAN_TRY(launch_walk(L, st, &n));
  PLAN_TRY(launch_row_scan(sd.R, w, st));
  if (p->pairs > 0) {
    PLAN_TRY(launch_gather(0, sd.R, w, p->out_i, p->out_j, p->out_w, L.a.unweighted,
                           p->pairs, st));
    PLAN_TRY(launch_localize(p->out_i, p->out_j, p->pairs, p->row_base, p->count, w.row_ptr,
                             p->offsets, st));
  } else {
    PLAN_TRY(cudaMemsetAsync(p->offsets, 0, sizeof(long long) * (p->count + 1), st));
  }
  if (launches) *launches = 1 + 2 + 1 + 4 + 1 + n + 3 + 2;
  return cudaSuccess;
}
#undef PLAN_TRY

}  // namespace
namespace {

// Validates the device input h as every call does and fills p with it and
// both sides' CSR->CSC maps, written to map0 and map1 (device arrays of nnz
// entries owned by the caller).  Synchronises `st`.
int prepare(const slg_hypergraph *h, int32_t *map0, int32_t *map1, cudaStream_t st,
            Prepared *p) {
  int rc = check_args(h, 1, 0);
  if (rc != SLG_OK) return rc;
  const Side sd = side_of(h, 0);
  Pool pool(st);
  Meta *meta = nullptr;
  SLG_TRY(pool.get(&meta, 1));
  SLG_TRY(cudaMemsetAsync(meta, 0, sizeof(Meta), st));
  SLG_TRY(launch_validate(sd, meta, st));
  SLG_TRY(launch_csr2csc(sd, map0, meta, st));
  Meta *mh = nullptr, *mv = nullptr;
  SLG_TRY(thread_meta(&mh, &mv));
  SLG_TRY(launch_meta_copy(meta, mv, st));
  SLG_TRY(cudaStreamSynchronize(st));
  if (mh->err) {
    t_err_where = mh->err_where;
    return mh->err;
  }
  // the input is valid: map0 is a permutation of [0, nnz)
  SLG_TRY(launch_invert(map0, h->nnz, map1, st));
  SLG_TRY(cudaStreamSynchronize(st));
  p->h = *h;
  p->map[0] = map0;
  p->map[1] = map1;
  return SLG_OK;
}

// Device copy of a host hypergraph, enqueued on `st` (buffers from `pool`).
int upload(const slg_hypergraph *hh, Pool &pool, cudaStream_t st, slg_hypergraph *d) {
  *d = *hh;
  int32_t *e_off, *e_idx, *v_off, *v_idx;
  const size_t m = (size_t)hh->n_edges, n = (size_t)hh->n_vertices, nnz = (size_t)hh->nnz;
  SLG_TRY(pool.get(&e_off, m + 1));
  SLG_TRY(pool.get(&v_off, n + 1));
  SLG_TRY(pool.get(&e_idx, nnz));
  SLG_TRY(pool.get(&v_idx, nnz));
  SLG_TRY(cudaMemcpyAsync(e_off, hh->e_off, (m + 1) * 4, cudaMemcpyHostToDevice, st));
  SLG_TRY(cudaMemcpyAsync(v_off, hh->v_off, (n + 1) * 4, cudaMemcpyHostToDevice, st));
  if (nnz) {
    SLG_TRY(cudaMemcpyAsync(e_idx, hh->e_idx, nnz * 4, cudaMemcpyHostToDevice, st));
    SLG_TRY(cudaMemcpyAsync(v_idx, hh->v_idx, nnz * 4, cudaMemcpyHostToDevice, st));
  }
  d->e_off = e_off;
  d->e_idx = e_idx;
  d->v_off = v_off;
  d->v_idx = v_idx;
  return SLG_OK;
}

// One query of slg_build_host_many / slg_build_host_csr: device outputs
// from the library pool on `st`, the build, then the copies back on `cs`
// once the build is done (the device buffers are released on `cs` after
// them).  Returns the query's status.
int host_query(const slg_hypergraph *d, slg_query *q, cudaStream_t st, cudaStream_t cs,
               cudaEvent_t done, std::vector<void *> *keep, int32_t *bad) {
  q->n_pairs = 0;
  if (q->flags & SLG_ASYNC) return SLG_ERR_INVALID;
  const bool unweighted = (q->flags & SLG_UNWEIGHTED) != 0;
  // SLG_W16: the weights are narrowed on the device (into buf[4]) and
  // copied back as uint16; *bad is set when one does not fit
  const bool w16 = (q->flags & SLG_W16) != 0 && !unweighted;
  const uint32_t flags = q->flags & ~(uint32_t)SLG_W16;
  const bool rows_form = q->row_ptr != nullptr;
  if (q->capacity < 0) return SLG_ERR_INVALID;
  if (q->capacity > 0 &&
      ((!rows_form && !q->out_i) || !q->out_j || (!unweighted && !q->out_w)))
    return SLG_ERR_INVALID;
  const int32_t R = (flags & SLG_DUAL) ? d->n_vertices : d->n_edges;
  cudaMemPool_t mem = lib_pool();
  void *buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  auto alloc = [&](int k, size_t bytes) {
    bytes = bytes < 16 ? 16 : bytes;
    cudaError_t e = mem ? cudaMallocFromPoolAsync(&buf[k], bytes, mem, st)
                        : cudaMallocAsync(&buf[k], bytes, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      buf[k] = nullptr;
    }
    return e;
  };
  auto release = [&](cudaStream_t on) {
    for (void *b : buf)
      if (b) cudaFreeAsync(b, on);
  };
  const size_t cap = (size_t)q->capacity;
  cudaError_t e = cudaSuccess;
  if (cap > 0) {
    if (!rows_form) e = alloc(0, cap * 4);
    if (e == cudaSuccess) e = alloc(1, cap * 4);
    if (e == cudaSuccess && !unweighted) e = alloc(2, cap * 4);
  }
  if (e == cudaSuccess && rows_form) e = alloc(3, ((size_t)R + 1) * 8);
  if (e == cudaSuccess && w16 && cap > 0) e = alloc(4, cap * 2);
  if (e != cudaSuccess) {
    release(st);
    return status_of(e);
  }
  int64_t pairs = 0;
  int rc = run(d, q->s, flags, 0, R, kOpBuild, static_cast<int32_t *>(buf[0]),
               static_cast<int32_t *>(buf[1]), static_cast<int32_t *>(buf[2]), q->capacity,
               &pairs, st, nullptr, nullptr, static_cast<long long *>(buf[3]));
  q->n_pairs = pairs;
  if (rc != SLG_OK) {
    release(st);
    return rc;
  }
  if (w16 && pairs > 0 &&
      launch_pack_w16(static_cast<const int32_t *>(buf[2]), pairs,
                      static_cast<uint16_t *>(buf[4]), bad, st) != cudaSuccess) {
    cudaGetLastError();
    release(st);
    return SLG_ERR_CUDA;
  }
  // the copies back wait for the build (the stream already synchronised
  // inside run; the event keeps the order explicit for the copy stream)
  if (cudaEventRecord(done, st) != cudaSuccess || cudaStreamWaitEvent(cs, done, 0) != cudaSuccess) {
    cudaGetLastError();
    release(st);
    return SLG_ERR_CUDA;
  }
  const size_t p = (size_t)pairs;
  cudaError_t c = cudaSuccess;
  if (rows_form)
    c = cudaMemcpyAsync(q->row_ptr, buf[3], ((size_t)R + 1) * 8, cudaMemcpyDeviceToHost, cs);
  if (p > 0) {
    if (c == cudaSuccess && !rows_form)
      c = cudaMemcpyAsync(q->out_i, buf[0], p * 4, cudaMemcpyDeviceToHost, cs);
    if (c == cudaSuccess) c = cudaMemcpyAsync(q->out_j, buf[1], p * 4, cudaMemcpyDeviceToHost, cs);
    if (c == cudaSuccess && !unweighted)
      c = w16 ? cudaMemcpyAsync(q->out_w, buf[4], p * 2, cudaMemcpyDeviceToHost, cs)
              : cudaMemcpyAsync(q->out_w, buf[2], p * 4, cudaMemcpyDeviceToHost, cs);
  }
  // the buffers stay until every copy of the call is done and are then
  // released on `st`, so that the pool hands them to the next call on `st`
  for (void *b : buf)
    if (b) keep->push_back(b);
  if (c != cudaSuccess) {
    cudaGetLastError();
    return SLG_ERR_CUDA;
  }
  return SLG_OK;
}

}  // namespace
}  // namespace slg

using namespace slg;

extern "C" {

int slg_count(const slg_hypergraph *h, int32_t s, uint32_t flags, int64_t *n_pairs,
              void *stream) {
  if (!h) return SLG_ERR_INVALID;
  const int32_t R = (flags & SLG_DUAL) ? h->n_vertices : h->n_edges;
  return run(h, s, flags, 0, R, kOpCount, nullptr, nullptr, nullptr, 0, n_pairs,
             (cudaStream_t)stream);
}

int slg_build(const slg_hypergraph *h, int32_t s, uint32_t flags, int32_t *out_i,
              int32_t *out_j, int32_t *out_w, int64_t capacity, int64_t *n_pairs,
              void *stream) {
  if (!h) return SLG_ERR_INVALID;
  const int32_t R = (flags & SLG_DUAL) ? h->n_vertices : h->n_edges;
  return run(h, s, flags, 0, R, kOpBuild, out_i, out_j, out_w, capacity, n_pairs,
             (cudaStream_t)stream);
}

int slg_build_rows(const slg_hypergraph *h, int32_t s, uint32_t flags, int32_t row_begin,
                   int32_t row_end, int32_t *out_i, int32_t *out_j, int32_t *out_w,
                   int64_t capacity, int64_t *n_pairs, void *stream) {
  return run(h, s, flags, row_begin, row_end, kOpBuild, out_i, out_j, out_w, capacity, n_pairs,
             (cudaStream_t)stream);
}

int slg_row_offsets(const slg_hypergraph *h, int32_t s, uint32_t flags, int64_t *row_ptr,
                    void *stream) {
  if (!h || !row_ptr) return SLG_ERR_INVALID;
  if ((flags & SLG_ALGO_MASK) != SLG_ALGO_BINNED ||
      (flags & (SLG_RELABEL_ASC | SLG_RELABEL_DESC)))
    return SLG_ERR_UNSUPPORTED;
  const int32_t R = (flags & SLG_DUAL) ? h->n_vertices : h->n_edges;
  int64_t pairs = 0;
  return run(h, s, flags, 0, R, kOpCount, nullptr, nullptr, nullptr, 0, &pairs,
             (cudaStream_t)stream, nullptr, nullptr, reinterpret_cast<long long *>(row_ptr));
}

int slg_row_work(const slg_hypergraph *h, int32_t s, uint32_t flags, int32_t *work,
                 int64_t *wedges, void *stream) {
  if (!h || !work || !wedges) return SLG_ERR_INVALID;
  if ((flags & SLG_ALGO_MASK) != SLG_ALGO_BINNED || (flags & (SLG_RELABEL_ASC | SLG_RELABEL_DESC)))
    return SLG_ERR_UNSUPPORTED;
  const int32_t R = (flags & SLG_DUAL) ? h->n_vertices : h->n_edges;
  return run(h, s, flags, 0, R, kOpWedges, nullptr, nullptr, nullptr, 0, wedges,
             (cudaStream_t)stream, nullptr, nullptr, nullptr, work);
}

int slg_wedges(const slg_hypergraph *h, int32_t s, uint32_t flags, int64_t *wedges,
               void *stream) {
  if (!h) return SLG_ERR_INVALID;
  const int32_t R = (flags & SLG_DUAL) ? h->n_vertices : h->n_edges;
  return run(h, s, flags, 0, R, kOpWedges, nullptr, nullptr, nullptr, 0, wedges,
             (cudaStream_t)stream);
}

int slg_build_host(const slg_hypergraph *hh, int32_t s, uint32_t flags, int32_t *out_i,
                   int32_t *out_j, int32_t *out_w, int64_t capacity, int64_t *n_pairs,
                   void *stream) {
  const bool async = (flags & SLG_ASYNC) != 0;
  flags &= ~(uint32_t)SLG_ASYNC;
  int rc = check_args(hh, s, flags);
  if (rc != SLG_OK) return rc;
  if (!n_pairs || capacity < 0) return SLG_ERR_INVALID;
  const bool unweighted = (flags & SLG_UNWEIGHTED) != 0;
  if (capacity > 0 && (!out_i || !out_j || (!unweighted && !out_w))) return SLG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  Pool pool(st);
  slg_hypergraph d;
  rc = upload(hh, pool, st, &d);
  if (rc != SLG_OK) return rc;
  int32_t *oi = nullptr, *oj = nullptr, *ow = nullptr;
  if (capacity > 0) {
    SLG_TRY(pool.get(&oi, (size_t)capacity));
    SLG_TRY(pool.get(&oj, (size_t)capacity));
    if (!unweighted) SLG_TRY(pool.get(&ow, (size_t)capacity));
  }
  int64_t pairs = 0;
  rc = slg_build(&d, s, flags, oi, oj, ow, capacity, &pairs, stream);
  *n_pairs = pairs;
  if (rc != SLG_OK) return rc;
  if (pairs > 0) {
    SLG_TRY(cudaMemcpyAsync(out_i, oi, (size_t)pairs * 4, cudaMemcpyDeviceToHost, st));
    SLG_TRY(cudaMemcpyAsync(out_j, oj, (size_t)pairs * 4, cudaMemcpyDeviceToHost, st));
    if (!unweighted)
      SLG_TRY(cudaMemcpyAsync(out_w, ow, (size_t)pairs * 4, cudaMemcpyDeviceToHost, st));
  }
  // the device buffers are released after the copies, in stream order
  if (!async) SLG_TRY(cudaStreamSynchronize(st));
  return SLG_OK;
}

int slg_build_csr(const slg_hypergraph *h, int32_t s, uint32_t flags, int64_t *row_ptr,
                  int32_t *out_j, int32_t *out_w, int64_t capacity, int64_t *n_pairs,
                  void *stream) {
  if (!h || !row_ptr) return SLG_ERR_INVALID;
  const int32_t R = (flags & SLG_DUAL) ? h->n_vertices : h->n_edges;
  return run(h, s, flags, 0, R, kOpBuild, nullptr, out_j, out_w, capacity, n_pairs,
             (cudaStream_t)stream, nullptr, nullptr, reinterpret_cast<long long *>(row_ptr));
}

int slg_build_host_many(const slg_hypergraph *hh, slg_query *queries, int32_t count,
                        void *stream) {
  if (!queries || count < 0) return SLG_ERR_INVALID;
  for (int32_t k = 0; k < count; ++k) {
    queries[k].status = SLG_ERR_INVALID;
    queries[k].n_pairs = 0;
  }
  if (count == 0) return SLG_OK;
  int rc = check_args(hh, 1, 0);
  if (rc != SLG_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Pool pool(st);
  slg_hypergraph d;
  rc = upload(hh, pool, st, &d);
  if (rc != SLG_OK) return rc;
  // validated and mapped once for every query of the call
  Prepared prep;
  int32_t *map0 = nullptr, *map1 = nullptr;
  SLG_TRY(pool.get(&map0, (size_t)std::max<int64_t>(d.nnz, 1)));
  SLG_TRY(pool.get(&map1, (size_t)std::max<int64_t>(d.nnz, 1)));
  rc = prepare(&d, map0, map1, st, &prep);
  if (rc != SLG_OK) {
    for (int32_t k = 0; k < count; ++k) queries[k].status = rc;
    return rc;
  }
  PrepScope prep_scope(&prep);
  int dev = 0;
  cudaStream_t cs = nullptr;
  cudaEvent_t done = nullptr;
  SLG_TRY(cudaGetDevice(&dev));
  SLG_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    cudaStreamDestroy(cs);
    return SLG_ERR_CUDA;
  }
  // one flag per query: a weight too large for SLG_W16
  int32_t *bad = nullptr;
  cudaError_t eb = pool.get(&bad, (size_t)count);
  if (eb == cudaSuccess) eb = cudaMemsetAsync(bad, 0, sizeof(int32_t) * (size_t)count, st);
  if (eb != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(done);
    cudaStreamDestroy(cs);
    return status_of(eb);
  }
  int first = SLG_OK;
  std::vector<void *> keep;
  for (int32_t k = 0; k < count; ++k) {
    const int q = host_query(&d, &queries[k], st, cs, done, &keep, bad + k);
    queries[k].status = q;
  }
  // every copy back done, then the device outputs and the uploaded input
  // (Pool) are released on `st`
  cudaError_t e1 = cudaEventRecord(done, cs);
  if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(st, done, 0);
  for (void *b : keep) cudaFreeAsync(b, st);
  std::vector<int32_t> bad_h((size_t)count, 0);
  const cudaError_t e3 = cudaMemcpyAsync(bad_h.data(), bad, sizeof(int32_t) * (size_t)count,
                                         cudaMemcpyDeviceToHost, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  cudaEventDestroy(done);
  cudaStreamDestroy(cs);
  if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
    cudaGetLastError();
    return SLG_ERR_CUDA;
  }
  for (int32_t k = 0; k < count; ++k) {
    if (queries[k].status == SLG_OK && bad_h[k]) queries[k].status = SLG_ERR_UNSUPPORTED;
    if (queries[k].status != SLG_OK && first == SLG_OK) first = queries[k].status;
  }
  return first;
}

int slg_build_host_csr(const slg_hypergraph *hh, int32_t s, uint32_t flags, int64_t *row_ptr,
                       int32_t *out_j, int32_t *out_w, int64_t capacity, int64_t *n_pairs,
                       void *stream) {
  if (!row_ptr || !n_pairs) return SLG_ERR_INVALID;
  slg_query q = {};
  q.s = s;
  q.flags = flags;
  q.row_ptr = row_ptr;
  q.out_j = out_j;
  q.out_w = out_w;
  q.capacity = capacity;
  const int rc = slg_build_host_many(hh, &q, 1, stream);
  *n_pairs = q.n_pairs;
  return rc != SLG_OK ? rc : q.status;
}

int slg_filter(const int32_t *in_i, const int32_t *in_j, const int32_t *in_w, int64_t n,
               int32_t s, int32_t *out_i, int32_t *out_j, int32_t *out_w, int64_t capacity,
               int64_t *n_pairs, void *stream) {
  if (!n_pairs || n < 0 || s < 1 || capacity < 0) return SLG_ERR_INVALID;
  if (n > 0 && (!in_i || !in_j || !in_w)) return SLG_ERR_INVALID;
  if (capacity > 0 && (!out_i || !out_j)) return SLG_ERR_INVALID;
  *n_pairs = 0;
  if (n == 0) return SLG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  Pool pool(st);
  long long *tile = nullptr;
  const int64_t nt = keep_tiles(n);
  SLG_TRY(pool.get(&tile, (size_t)nt + 1));
  SLG_TRY(launch_keep_count(in_w, n, s, tile, st));
  long long total = 0;
  SLG_TRY(cudaMemcpyAsync(&total, tile + nt, sizeof(long long), cudaMemcpyDeviceToHost, st));
  SLG_TRY(cudaStreamSynchronize(st));
  *n_pairs = total;
  if (total > capacity) return SLG_ERR_CAPACITY;
  if (total > 0) SLG_TRY(launch_keep_write(in_i, in_j, in_w, n, s, tile, out_i, out_j, out_w, st));
  SLG_TRY(cudaStreamSynchronize(st));
  return SLG_OK;
}

int slg_build_sweep(const slg_hypergraph *h, const int32_t *s, int32_t count, uint32_t flags,
                    int32_t *const *out_i, int32_t *const *out_j, int32_t *const *out_w,
                    const int64_t *capacity, int64_t *n_pairs, void *stream) {
  if (!h || !s || count < 1 || count > 64 || !out_i || !out_j || !out_w || !capacity ||
      !n_pairs)
    return SLG_ERR_INVALID;
  if (flags & SLG_UNWEIGHTED) return SLG_ERR_UNSUPPORTED;  // the weights decide membership
  int32_t k0 = 0;
  for (int32_t k = 0; k < count; ++k) {
    if (s[k] < 1) return SLG_ERR_INVALID;
    n_pairs[k] = -1;
    if (s[k] < s[k0]) k0 = k;
  }
  // L_{s_min} by one walk, into the caller's list of the smallest threshold
  if (capacity[k0] > 0 && !out_w[k0]) return SLG_ERR_INVALID;
  int rc = slg_build(h, s[k0], flags, out_i[k0], out_j[k0], out_w[k0], capacity[k0],
                     &n_pairs[k0], stream);
  if (rc != SLG_OK) return rc;
  const slg_stats base_stats = t_stats;
  const int64_t n0 = n_pairs[k0];
  cudaStream_t st = (cudaStream_t)stream;
  int result = SLG_OK;
  for (int32_t k = 0; k < count; ++k) {
    if (k == k0) continue;
    if (s[k] == s[k0]) {  // the same list
      n_pairs[k] = n0;
      if (n0 > capacity[k]) {
        result = SLG_ERR_CAPACITY;
        continue;
      }
      if (n0 > 0) {
        if (!out_i[k] || !out_j[k]) return SLG_ERR_INVALID;
        SLG_TRY(cudaMemcpyAsync(out_i[k], out_i[k0], (size_t)n0 * 4, cudaMemcpyDeviceToDevice, st));
        SLG_TRY(cudaMemcpyAsync(out_j[k], out_j[k0], (size_t)n0 * 4, cudaMemcpyDeviceToDevice, st));
        if (out_w[k])
          SLG_TRY(cudaMemcpyAsync(out_w[k], out_w[k0], (size_t)n0 * 4, cudaMemcpyDeviceToDevice,
                                  st));
      }
      continue;
    }
    rc = slg_filter(out_i[k0], out_j[k0], out_w[k0], n0, s[k], out_i[k], out_j[k], out_w[k],
                    capacity[k], &n_pairs[k], stream);
    if (rc == SLG_ERR_CAPACITY) result = rc;
    else if (rc != SLG_OK) return rc;
  }
  SLG_TRY(cudaStreamSynchronize(st));
  t_stats = base_stats;
  return result;
}

// Device check of a pair list; returns SLG_OK or SLG_ERR_INVALID (synchronises).
static int check_pairs(const int32_t *a, const int32_t *b, int64_t n, int32_t R, int canonical,
                       Pool &pool, cudaStream_t st) {
  if (n == 0) return SLG_OK;
  int32_t *err = nullptr;
  SLG_TRY(pool.get(&err, 1));
  SLG_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
  SLG_TRY(launch_check_pairs(a, b, n, R, canonical, err, st));
  int32_t h = 0;
  SLG_TRY(cudaMemcpyAsync(&h, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SLG_TRY(cudaStreamSynchronize(st));
  return h ? SLG_ERR_INVALID : SLG_OK;
}

int slg_squeeze(const int32_t *in_i, const int32_t *in_j, int64_t n, int32_t R, int32_t *out_i,
                int32_t *out_j, int32_t *old_of_new, int32_t *n_ids, void *stream) {
  if (!n_ids || n < 0 || R < 0 || (n > 0 && (!in_i || !in_j || !out_i || !out_j)) ||
      (R > 0 && !old_of_new))
    return SLG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  Pool pool(st);
  int rc = check_pairs(in_i, in_j, n, R, 0, pool, st);
  if (rc) return rc;
  int32_t *mark, *rank, *tile;
  SLG_TRY(pool.get(&mark, (size_t)R + 1));
  SLG_TRY(pool.get(&rank, (size_t)R + 1));
  SLG_TRY(pool.get(&tile, (size_t)xscan_tiles((int64_t)R + 1) + 1));
  SLG_TRY(cudaMemsetAsync(mark, 0, ((size_t)R + 1) * sizeof(int32_t), st));
  SLG_TRY(launch_mark(in_i, in_j, n, mark, st));
  SLG_TRY(launch_xscan(mark, rank, (int64_t)R + 1, tile, st));
  SLG_TRY(launch_squeeze(in_i, in_j, n, R, mark, rank, out_i, out_j, old_of_new, st));
  int32_t ids = 0;
  SLG_TRY(cudaMemcpyAsync(&ids, rank + R, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SLG_TRY(cudaStreamSynchronize(st));
  *n_ids = ids;
  return SLG_OK;
}

int slg_adjacency(const int32_t *in_i, const int32_t *in_j, const int32_t *in_w, int64_t n,
                  int32_t V, int64_t *adj_off, int32_t *adj, int32_t *adj_w, void *stream) {
  if (n < 0 || V < 0 || n >= ((int64_t)1 << 30) || !adj_off ||
      (n > 0 && (!in_i || !in_j || !adj || (adj_w && !in_w))))
    return SLG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  Pool pool(st);
  int rc = check_pairs(in_i, in_j, n, V, 1, pool, st);
  if (rc) return rc;
  int32_t *up, *lo;
  SLG_TRY(pool.get(&up, (size_t)V + 1));
  SLG_TRY(pool.get(&lo, (size_t)V + 1));
  SLG_TRY(cudaMemsetAsync(up, 0, ((size_t)V + 1) * sizeof(int32_t), st));
  SLG_TRY(cudaMemsetAsync(lo, 0, ((size_t)V + 1) * sizeof(int32_t), st));
  long long *off = reinterpret_cast<long long *>(adj_off);
  SLG_TRY(launch_adjacency_offsets(in_i, in_j, n, V, up, lo, off, st));
  if (n > 0) {
    long long *first, *lfirst;
    uint32_t *keys, *keys_tmp;
    int32_t *pos, *pos_tmp, *hist;
    SLG_TRY(pool.get(&first, (size_t)V + 1));
    SLG_TRY(pool.get(&lfirst, (size_t)V + 1));
    SLG_TRY(pool.get(&keys, (size_t)n));
    SLG_TRY(pool.get(&keys_tmp, (size_t)n));
    SLG_TRY(pool.get(&pos, (size_t)n));
    SLG_TRY(pool.get(&pos_tmp, (size_t)n));
    SLG_TRY(pool.get(&hist, radix_sort_scratch_ints(n)));
    SLG_TRY(launch_adjacency_fill(in_i, in_j, in_w, n, V, off, lo, first, lfirst, keys,
                                  keys_tmp, pos, pos_tmp, hist, adj, adj_w, st));
  }
  SLG_TRY(cudaStreamSynchronize(st));
  return SLG_OK;
}

int slg_components(const int32_t *in_i, const int32_t *in_j, int64_t n, int32_t R,
                   int32_t *labels, int64_t *n_components, void *stream) {
  if (!n_components || n < 0 || R < 0 || R > kComponentsMaxR || (n > 0 && (!in_i || !in_j)) ||
      (R > 0 && !labels))
    return SLG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  Pool pool(st);
  int rc = check_pairs(in_i, in_j, n, R, 0, pool, st);
  if (rc) return rc;
  int32_t *mark, *err;
  unsigned long long *cnt;
  SLG_TRY(pool.get(&mark, (size_t)R + 1));
  SLG_TRY(pool.get(&err, 1));
  SLG_TRY(pool.get(&cnt, 1));
  SLG_TRY(cudaMemsetAsync(mark, 0, ((size_t)R + 1) * sizeof(int32_t), st));
  SLG_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
  SLG_TRY(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
  SLG_TRY(launch_mark(in_i, in_j, n, mark, st));
  SLG_TRY(launch_components(in_i, in_j, n, R, labels, mark, cnt, err, st));
  unsigned long long hc = 0;
  int32_t he = 0;
  SLG_TRY(cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, st));
  SLG_TRY(cudaMemcpyAsync(&he, err, sizeof(he), cudaMemcpyDeviceToHost, st));
  SLG_TRY(cudaStreamSynchronize(st));
  if (he) return SLG_ERR_TIMEOUT;  // a bounded loop gave up (not expected)
  *n_components = (int64_t)hc;
  return SLG_OK;
}

int slg_tile_overlap(const uint8_t *A, int32_t rows_pad, int32_t cols_pad, int32_t *C,
                     void *stream) {
  if (!A || !C || rows_pad <= 0 || cols_pad <= 0 || rows_pad % 128 || cols_pad % 128 ||
      cols_pad >= (1 << 24) || (reinterpret_cast<uintptr_t>(A) & 15))
    return SLG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  Pool pool(st);
  const int64_t nt = rows_pad / 128;
  void *tasks = nullptr;
  int32_t *err = nullptr;
  SLG_TRY(pool.get(reinterpret_cast<int64_t **>(&tasks), (size_t)(nt * (nt + 1) / 2)));
  SLG_TRY(pool.get(&err, 1));
  SLG_TRY(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
  Events evs(t_profile != 0);
  if (evs.on) cudaEventRecord(evs.ev[kEvTile0], st);
  cudaError_t e = launch_tile_overlap(A, rows_pad, cols_pad, C, tasks, err, st);
  if (evs.on) cudaEventRecord(evs.ev[kEvTile1], st);
  if (e == cudaErrorNotSupported) return SLG_ERR_UNSUPPORTED;
  if (e == cudaErrorInvalidValue) return SLG_ERR_INVALID;
  SLG_TRY(e);
  int32_t h_err = 0;
  SLG_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SLG_TRY(cudaStreamSynchronize(st));
  slg_stats stats = {};
  if (evs.on) {
    stats.profiled = 1;
    stats.ms_tile = evs.ms(kEvTile0, kEvTile1);
  }
  t_stats = stats;
  return h_err ? SLG_ERR_TIMEOUT : SLG_OK;
}

int slg_release_memory(void) {
  cudaMemPool_t m = lib_pool();
  if (!m) return SLG_OK;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(m, 0) != cudaSuccess) {
    cudaGetLastError();
    return SLG_ERR_CUDA;
  }
  return SLG_OK;
}

int slg_set_core_params(int32_t tau_c, int32_t tau_r, float min_density) {
  if (tau_c < 1 || tau_r < 1 || !(min_density > 0.f && min_density <= 1.f))
    return SLG_ERR_INVALID;
  t_tau_c = tau_c;
  t_tau_r = tau_r;
  t_min_density = min_density;
  return SLG_OK;
}

int slg_set_profiling(int enable) {
  t_profile = enable ? 1 : 0;
  return SLG_OK;
}

int slg_last_stats(slg_stats *out) {
  if (!out) return SLG_ERR_INVALID;
  *out = t_stats;
  return SLG_OK;
}

const char *slg_strerror(int status) {
  switch (status) {
    case SLG_OK: return "ok";
    case SLG_ERR_INVALID: return "invalid argument or malformed incidence";
    case SLG_ERR_CAPACITY: return "output capacity smaller than the pair count";
    case SLG_ERR_NOMEM: return "device memory allocation failed";
    case SLG_ERR_CUDA: return "CUDA runtime error";
    case SLG_ERR_TIMEOUT: return "bounded device wait gave up";
    case SLG_ERR_UNSUPPORTED: return "unsupported flag combination or size";
    case SLG_ERR_TOO_LARGE: return "input too large for the fixed working memory of slg_count_noalloc";
    default: return "unknown status";
  }
}

int slg_abi_version(void) { return SLG_ABI_VERSION; }

int slg_last_error_where(void) { return t_err_where; }

}  // extern "C"

extern "C" int slg_plan_create(const slg_hypergraph *hs, const int32_t *s, int32_t count,
                               uint32_t flags, slg_plan **plan_out, void *stream) {
  if (!hs || !s || count < 1 || !plan_out) return SLG_ERR_INVALID;
  if (flags & ~(uint32_t)(SLG_DUAL | SLG_UNWEIGHTED)) return SLG_ERR_UNSUPPORTED;
  *plan_out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  int64_t M = 0, N = 0, K = 0, max_len = 0;
  for (int32_t g = 0; g < count; ++g) {
    int rc = check_args(&hs[g], s[g], flags);
    if (rc != SLG_OK) return rc;
    M += hs[g].n_edges;
    N += hs[g].n_vertices;
    K += hs[g].nnz;
    max_len = std::max<int64_t>(max_len, std::max<int64_t>(hs[g].nnz,
                                                            std::max(hs[g].n_edges, hs[g].n_vertices)));
  }
  if (M >= (int64_t(1) << 31) || N >= (int64_t(1) << 31) || K >= (int64_t(1) << 31))
    return SLG_ERR_INVALID;
  std::unique_ptr<slg_plan> p(new slg_plan());
  cudaGetDevice(&p->dev);
  p->flags = flags;
  p->count = count;
  const bool dual = (flags & SLG_DUAL) != 0;
  // 1. the union
  int32_t *e_off, *e_idx, *v_off, *v_idx;
  SLG_TRY(p->mem.get(&e_off, (size_t)M + 1));
  SLG_TRY(p->mem.get(&v_off, (size_t)N + 1));
  SLG_TRY(p->mem.get(&e_idx, (size_t)K));
  SLG_TRY(p->mem.get(&v_idx, (size_t)K));
  SLG_TRY(p->mem.get(&p->row_s_e, (size_t)M + 1));
  SLG_TRY(p->mem.get(&p->row_s_v, (size_t)N + 1));
  SLG_TRY(p->mem.get(&p->row_fhi_e, (size_t)M + 1));
  SLG_TRY(p->mem.get(&p->row_fhi_v, (size_t)N + 1));
  std::vector<BatchGraph> bg((size_t)count);
  std::vector<int32_t> base((size_t)count + 1);
  int64_t eb = 0, vb = 0, kb = 0;
  for (int32_t g = 0; g < count; ++g) {
    bg[g] = BatchGraph{hs[g].e_off, hs[g].e_idx, hs[g].v_off, hs[g].v_idx, hs[g].n_edges,
                       hs[g].n_vertices, hs[g].nnz, (int32_t)eb, (int32_t)vb, kb, s[g]};
    base[g] = (int32_t)(dual ? vb : eb);
    eb += hs[g].n_edges;
    vb += hs[g].n_vertices;
    kb += hs[g].nnz;
  }
  base[count] = (int32_t)(dual ? vb : eb);
  BatchGraph *bg_d;
  SLG_TRY(p->mem.get(&bg_d, (size_t)count));
  SLG_TRY(p->mem.get(&p->row_base, (size_t)count + 1));
  SLG_TRY(cudaMemcpyAsync(bg_d, bg.data(), sizeof(BatchGraph) * count, cudaMemcpyHostToDevice, st));
  SLG_TRY(cudaMemcpyAsync(p->row_base, base.data(), sizeof(int32_t) * (count + 1),
                          cudaMemcpyHostToDevice, st));
  const int32_t tailv[1] = {(int32_t)K};
  SLG_TRY(cudaMemcpyAsync(e_off + M, tailv, 4, cudaMemcpyHostToDevice, st));
  SLG_TRY(cudaMemcpyAsync(v_off + N, tailv, 4, cudaMemcpyHostToDevice, st));
  SLG_TRY(launch_concat(bg_d, count, (int32_t)std::min<int64_t>(max_len, 1 << 30), e_off, e_idx,
                        v_off, v_idx, p->row_s_e, p->row_s_v, p->row_fhi_e, p->row_fhi_v,
                        st));
  SLG_TRY(cudaStreamSynchronize(st));
  p->u = slg_hypergraph{(int32_t)M, (int32_t)N, K, e_off, e_idx, v_off, v_idx};
  p->sd = side_of(&p->u, flags);
  p->sd.row_s = dual ? p->row_s_v : p->row_s_e;
  p->sd.row_fhi = dual ? p->row_fhi_v : p->row_fhi_e;
  // 2. sizes: one counting pass over the union (per-row thresholds)
  int64_t pairs = 0;
  int32_t max_work = 0;
  int rc = run(&p->u, 1, flags, 0, p->sd.R, kOpCount, nullptr, nullptr, nullptr, 0, &pairs, st,
               p->sd.row_s, &max_work, nullptr, nullptr, p->sd.row_fhi);
  if (rc != SLG_OK) return rc;
  p->pairs = pairs;
  // 3. persistent buffers
  Work &w = p->w;
  const int64_t nnz = K, R = p->sd.R;
  SLG_TRY(p->mem.get(&w.meta, 1));
  SLG_TRY(p->mem.get(&w.csr2csc, (size_t)nnz));
  SLG_TRY(p->mem.get(&w.qs, (size_t)nnz + 1));
  SLG_TRY(p->mem.get(&w.c_idx_s, (size_t)nnz + 1));
  SLG_TRY(p->mem.get(&w.c_off_s, (size_t)p->sd.C + 1));
  SLG_TRY(p->mem.get(&w.tail_beg, (size_t)nnz));
  SLG_TRY(p->mem.get(&w.tail_end, (size_t)nnz));
  SLG_TRY(p->mem.get(&w.tile, (size_t)((nnz + 4095) / 4096) + 1));
  SLG_TRY(p->mem.get(&w.bin_rows, (size_t)kNumBins * (R > 0 ? R : 1)));
  SLG_TRY(p->mem.get(&w.n_e, (size_t)R + 1));
  SLG_TRY(p->mem.get(&w.row_work, (size_t)R + 1));
  SLG_TRY(p->mem.get(&w.stage_pos, (size_t)R + 1));
  SLG_TRY(p->mem.get(&w.row_ptr, (size_t)R + 1));
  SLG_TRY(p->mem.get(&w.tile64, (size_t)((R + 4095) / 4096) + 1));
  SLG_TRY(p->mem.get(&w.stage_j, (size_t)std::max<int64_t>(pairs, 1)));
  SLG_TRY(p->mem.get(&w.stage_w, (size_t)std::max<int64_t>(pairs, 1)));
  w.stage_cap = pairs;
  SLG_TRY(p->mem.get(&p->out_i, (size_t)std::max<int64_t>(pairs, 1)));
  SLG_TRY(p->mem.get(&p->out_j, (size_t)std::max<int64_t>(pairs, 1)));
  SLG_TRY(p->mem.get(&p->out_w, (size_t)std::max<int64_t>(pairs, 1)));
  SLG_TRY(p->mem.get(&p->offsets, (size_t)count + 1));
  if (max_work > 0) {
    p->giant_stride = 4ll * max_work;
    SLG_TRY(p->mem.get(&p->giant, (size_t)giant_ctas() * (size_t)p->giant_stride));
  }
  // 4. autotuner: bin thresholds, timed on this batch
  // candidates: CTA-bin limits, the sparse bin's range (0: off) and the
  // dense-row ratio of the giant bin
  const Bins cands[] = {Bins{},
                        Bins{64, 1024, 4096},
                        Bins{128, 512, 4096},
                        Bins{128, 1024, 2048},
                        Bins{128, 1024, 4096, 8192},
                        Bins{128, 1024, 4096, 0},
                        Bins{128, 1024, 2048, 16384, 2048},
                        Bins{128, 1024, 4096, 16384, 4096, 4},
                        Bins{128, 1024, 4096, 16384, 4096, 16},
                        Bins{128, 1024, 4096, 16384, 4096, 8}};
  cudaEvent_t t0, t1;
  SLG_TRY(cudaEventCreate(&t0));
  SLG_TRY(cudaEventCreate(&t1));
  float best = 1e30f;
  Bins best_bins;
  for (const Bins &b : cands) {
    if (b.warp > kWarpMaxWork || b.ctas > kCtaSMaxWork || b.ctal > kCtaLMaxWork) continue;
    if (!p->giant && p->sd.R > 0 && max_work > b.ctal) continue;
    float ms = 0.f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(t0, st);
      cudaError_t e = enqueue_plan(p.get(), b, st, nullptr);
      cudaEventRecord(t1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      Meta *mh = nullptr;
      if (e == cudaSuccess) e = thread_meta(&mh);
      if (e == cudaSuccess) e = cudaMemcpy(mh, w.meta, sizeof(Meta), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        cudaGetLastError();
        return status_of(e);
      }
      // every candidate must reproduce the counted pairs exactly
      if (mh->err || mh->stage_overflow || (int64_t)mh->pairs != pairs) {
        if (debug_on())
          std::fprintf(stderr,
                       "slg: plan candidate %d/%d/%d: err %d at %d, staging overflow %llu, "
                       "pairs %llu, counted %lld\n",
                       b.warp, b.ctas, b.ctal, mh->err, mh->err_where, mh->stage_overflow,
                       mh->pairs, (long long)pairs);
        t_err_where = mh->err ? mh->err_where : kWhereStage;
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        return mh->err ? mh->err : SLG_ERR_INVALID;
      }
      float t = 0.f;
      cudaEventElapsedTime(&t, t0, t1);
      if (rep > 0) ms += t;  // first repetition warms up
    }
    if (ms < best) {
      best = ms;
      best_bins = b;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  p->bins = best_bins;
  p->tuned_ms = best / 2.f;
  // 5. capture the tuned build into a CUDA graph
  cudaStream_t cs;
  SLG_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = enqueue_plan(p.get(), p->bins, cs, &p->launches);
    e = cudaStreamEndCapture(cs, &p->graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    return status_of(e);
  }
  *plan_out = p.release();
  return SLG_OK;
}

extern "C" int slg_plan_execute(slg_plan *p, void *stream) {
  if (!p || !p->exec) return SLG_ERR_INVALID;
  cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return status_of(e);
  }
  return SLG_OK;
}

extern "C" int slg_plan_result(const slg_plan *p, const int32_t **out_i, const int32_t **out_j,
                               const int32_t **out_w, int64_t *n_pairs, int64_t *offsets) {
  if (!p) return SLG_ERR_INVALID;
  if (out_i) *out_i = p->out_i;
  if (out_j) *out_j = p->out_j;
  if (out_w) *out_w = (p->flags & SLG_UNWEIGHTED) ? nullptr : p->out_w;
  if (n_pairs) *n_pairs = p->pairs;
  if (offsets) {
    int32_t err = 0;
    cudaError_t e = cudaMemcpy(offsets, p->offsets, sizeof(long long) * (p->count + 1),
                               cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&err, &p->w.meta->err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return status_of(e);
    }
    if (err) return err;
  }
  return SLG_OK;
}

extern "C" int slg_plan_info(const slg_plan *p, int32_t *bins, float *tuned_ms,
                             int32_t *launches) {
  if (!p) return SLG_ERR_INVALID;
  if (bins) {
    bins[0] = p->bins.warp;
    bins[1] = p->bins.ctas;
    bins[2] = p->bins.ctal;
    bins[3] = p->bins.sparse;
    bins[4] = p->bins.bloom;
    bins[5] = p->bins.dense;
  }
  if (tuned_ms) *tuned_ms = p->tuned_ms;
  if (launches) *launches = p->launches;
  return SLG_OK;
}

extern "C" int slg_plan_destroy(slg_plan *p) {
  if (!p) return SLG_OK;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  delete p;
  return SLG_OK;
}

// ------------------------------------------------------------ graph handle --

struct slg_graph {
  slg::Prepared p;
  int32_t *maps = nullptr;  // both sides' CSR->CSC maps (2 x nnz)
  cudaStream_t st = nullptr;
  int dev = 0;
};

extern "C" int slg_graph_create(const slg_hypergraph *h, slg_graph **graph, void *stream) {
  if (!graph) return SLG_ERR_INVALID;
  *graph = nullptr;
  int rc = check_args(h, 1, 0);
  if (rc != SLG_OK) return rc;
  slg_graph *g = new (std::nothrow) slg_graph();
  if (!g) return SLG_ERR_NOMEM;
  g->st = (cudaStream_t)stream;
  cudaGetDevice(&g->dev);
  const size_t n = (size_t)std::max<int64_t>(h->nnz, 1);
  cudaMemPool_t mem = lib_pool();
  void *q = nullptr;
  const cudaError_t e = mem ? cudaMallocFromPoolAsync(&q, 2 * n * sizeof(int32_t), mem, g->st)
                            : cudaMallocAsync(&q, 2 * n * sizeof(int32_t), g->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete g;
    return status_of(e);
  }
  g->maps = static_cast<int32_t *>(q);
  rc = prepare(h, g->maps, g->maps + n, g->st, &g->p);
  if (rc != SLG_OK) {
    cudaFreeAsync(g->maps, g->st);
    cudaStreamSynchronize(g->st);
    delete g;
    return rc;
  }
  *graph = g;
  return SLG_OK;
}

namespace {
int graph_check(const slg_graph *g) {
  if (!g) return SLG_ERR_INVALID;
  int dev = 0;
  cudaGetDevice(&dev);
  return dev == g->dev ? SLG_OK : SLG_ERR_INVALID;
}
}  // namespace

extern "C" int slg_graph_count(const slg_graph *g, int32_t s, uint32_t flags, int64_t *n_pairs,
                               void *stream) {
  const int rc = graph_check(g);
  if (rc != SLG_OK) return rc;
  PrepScope scope(&g->p);
  return slg_count(&g->p.h, s, flags, n_pairs, stream);
}

extern "C" int slg_graph_build(const slg_graph *g, int32_t s, uint32_t flags, int32_t *out_i,
                               int32_t *out_j, int32_t *out_w, int64_t capacity,
                               int64_t *n_pairs, void *stream) {
  const int rc = graph_check(g);
  if (rc != SLG_OK) return rc;
  PrepScope scope(&g->p);
  return slg_build(&g->p.h, s, flags, out_i, out_j, out_w, capacity, n_pairs, stream);
}

extern "C" int slg_graph_destroy(slg_graph *g) {
  if (!g) return SLG_OK;
  cudaFreeAsync(g->maps, g->st);
  const cudaError_t e = cudaStreamSynchronize(g->st);
  delete g;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return SLG_ERR_CUDA;
  }
  return SLG_OK;
}
