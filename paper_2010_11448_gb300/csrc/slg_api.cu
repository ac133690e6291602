// C ABI of the slg library (declared in include/slg.h): argument checks,
// per-call working memory, the sequence of planning, walking and output
// kernels, and the single device->host read of the pair count.
#include <mutex>
#include <vector>

#include "slg_internal.cuh"

namespace slg {
namespace {

constexpr int kMaxDevices = 64;

// Per-device state kept between calls: the giant bin's dense counters (all
// zero between calls; the kernels restore the zeros they disturb) and a
// pinned copy of the Meta record.
struct DeviceCtx {
  std::mutex mu;
  int32_t *giant = nullptr;
  size_t giant_elems = 0;
  Meta *meta_host = nullptr;
  bool pool_ready = false;
};

DeviceCtx g_ctx[kMaxDevices];
thread_local slg_stats t_stats;
thread_local int t_profile = 0;

// Events of one profiled call: plan start, walk (kNumBins + 1), scan end,
// gather end.
struct Events {
  cudaEvent_t ev[kNumBins + 5] = {};
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
              kEvGather1 = kNumBins + 4;

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return SLG_OK;
  if (e == cudaErrorMemoryAllocation) return SLG_ERR_NOMEM;
  return SLG_ERR_CUDA;
}

// Stream-ordered allocations released (stream-ordered) when the call ends.
struct Pool {
  cudaStream_t st;
  std::vector<void *> ptrs;
  explicit Pool(cudaStream_t s) : st(s) {}
  template <class T>
  cudaError_t get(T **p, size_t count) {
    size_t bytes = count * sizeof(T);
    if (bytes < 16) bytes = 16;
    void *q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, bytes, st);
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

#define SLG_TRY(expr)                         \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) {                  \
      cudaGetLastError();                     \
      return status_of(_e);                   \
    }                                         \
  } while (0)

int check_args(const slg_hypergraph *h, int32_t s, uint32_t flags) {
  if (!h || s < 1) return SLG_ERR_INVALID;
  if (h->n_edges < 0 || h->n_vertices < 0 || h->nnz < 0 || h->nnz >= (int64_t(1) << 31))
    return SLG_ERR_INVALID;
  if (!h->e_off || !h->v_off) return SLG_ERR_INVALID;
  if (h->nnz > 0 && (!h->e_idx || !h->v_idx)) return SLG_ERR_INVALID;
  if ((flags & SLG_ALGO_MASK) != SLG_ALGO_BINNED) return SLG_ERR_UNSUPPORTED;
  if (flags & ~(uint32_t)(SLG_DUAL | SLG_UNWEIGHTED | SLG_ALGO_MASK)) return SLG_ERR_INVALID;
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

DeviceCtx &ctx_for_current(int *dev_out) {
  int dev = 0;
  cudaGetDevice(&dev);
  *dev_out = dev;
  return g_ctx[dev % kMaxDevices];
}

// Freed pool memory stays with the process instead of going back to the
// driver after every call.
void ensure_pool(DeviceCtx &c, int dev) {
  if (c.pool_ready) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  c.pool_ready = true;
}

cudaError_t ensure_giant(DeviceCtx &c, size_t elems, cudaStream_t st) {
  if (c.giant_elems >= elems) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  if (c.giant) cudaFree(c.giant);
  c.giant = nullptr;
  c.giant_elems = 0;
  e = cudaMalloc(&c.giant, elems * sizeof(int32_t));
  if (e != cudaSuccess) return e;
  e = cudaMemset(c.giant, 0, elems * sizeof(int32_t));
  if (e != cudaSuccess) return e;
  c.giant_elems = elems;
  return cudaSuccess;
}

enum Op { kOpCount, kOpBuild, kOpWedges };

// The whole pipeline for one side, one s and one row range.
int run(const slg_hypergraph *h, int32_t smin, uint32_t flags, int32_t row_begin,
        int32_t row_end, Op op, int32_t *out_i, int32_t *out_j, int32_t *out_w,
        int64_t capacity, int64_t *result, cudaStream_t st) {
  int rc = check_args(h, smin, flags);
  if (rc != SLG_OK) return rc;
  if (!result) return SLG_ERR_INVALID;
  const Side sd = side_of(h, flags);
  if (row_begin < 0 || row_end < row_begin || row_end > sd.R) return SLG_ERR_INVALID;
  const bool unweighted = (flags & SLG_UNWEIGHTED) != 0;
  if (op == kOpBuild) {
    if (capacity < 0) return SLG_ERR_INVALID;
    if (capacity > 0 && (!out_i || !out_j || (!unweighted && !out_w))) return SLG_ERR_INVALID;
  }
  const int32_t rows = row_end - row_begin;
  const int64_t nnz = sd.nnz;
  const int32_t R_pad = (int32_t)(((int64_t)sd.R + 1023) / 1024 * 1024);
  if (giant_smem_bytes(R_pad > 0 ? R_pad : 1024) > 200 * 1024) return SLG_ERR_UNSUPPORTED;

  int dev = 0;
  DeviceCtx &c = ctx_for_current(&dev);
  std::lock_guard<std::mutex> lock(c.mu);
  ensure_pool(c, dev);
  if (!c.meta_host) SLG_TRY(cudaMallocHost(&c.meta_host, sizeof(Meta)));

  slg_stats stats = {};
  int32_t launches = 0;
  Events evs(t_profile != 0 && op != kOpWedges);
  Pool pool(st);
  Work w = {};
  const int32_t ntiles = (int32_t)((nnz + 4095) / 4096);
  const int32_t ntiles64 = (rows + 4095) / 4096;
  SLG_TRY(pool.get(&w.meta, 1));
  SLG_TRY(pool.get(&w.csr2csc, (size_t)nnz));
  SLG_TRY(pool.get(&w.qs, (size_t)nnz + 1));
  SLG_TRY(pool.get(&w.c_idx_s, (size_t)nnz));
  SLG_TRY(pool.get(&w.c_off_s, (size_t)sd.C + 1));
  SLG_TRY(pool.get(&w.tail_beg, (size_t)nnz));
  SLG_TRY(pool.get(&w.tile, (size_t)ntiles + 1));
  SLG_TRY(pool.get(&w.bin_rows, (size_t)kNumBins * (rows > 0 ? rows : 1)));
  SLG_TRY(pool.get(&w.n_e, (size_t)rows + 1));
  SLG_TRY(pool.get(&w.stage_pos, (size_t)rows + 1));
  SLG_TRY(pool.get(&w.row_ptr, (size_t)rows + 1));
  SLG_TRY(pool.get(&w.tile64, (size_t)ntiles64 + 1));
  SLG_TRY(cudaMemsetAsync(w.meta, 0, sizeof(Meta), st));

  // Planning: validation, CSR->CSC map, filtered CSC, tails, work, bins.
  if (evs.on) cudaEventRecord(evs.ev[kEvPlan], st);
  SLG_TRY(launch_validate(sd, w.meta, st));
  SLG_TRY(launch_csr2csc(sd, w.csr2csc, w.meta, st));
  SLG_TRY(launch_filter(sd, smin, w, st));
  SLG_TRY(launch_rows_work(sd, smin, row_begin, row_end, w, st));
  launches += 2 + 1 + 4 + (rows > 0 ? 1 : 0);

  int64_t pairs = 0;
  if (op != kOpWedges) {
    // Staging for the single-walk build: sized by the caller's capacity; if
    // it cannot be had the rows that do not fit are re-walked directly.
    if (op == kOpBuild && capacity > 0) {
      if (pool.get(&w.stage_j, (size_t)capacity) == cudaSuccess &&
          (unweighted || pool.get(&w.stage_w, (size_t)capacity) == cudaSuccess)) {
        w.stage_cap = capacity;
      } else {
        w.stage_cap = 0;
      }
    }
    const int32_t gctas = giant_ctas_for_device();
    SLG_TRY(ensure_giant(c, (size_t)gctas * (size_t)R_pad, st));
    WalkLaunch L = {};
    L.w.r_off = sd.r_off;
    L.w.r_idx = sd.r_idx;
    L.w.c_off_s = w.c_off_s;
    L.w.c_idx_s = w.c_idx_s;
    L.w.tail_beg = w.tail_beg;
    L.a.mode = (op == kOpBuild) ? kStage : kCount;
    L.a.unweighted = unweighted;
    L.a.smin = smin;
    L.a.row_begin = row_begin;
    L.a.n_e = w.n_e;
    L.a.stage_pos = w.stage_pos;
    L.a.stage_j = w.stage_j;
    L.a.stage_w = w.stage_w;
    L.a.stage_cap = w.stage_cap;
    L.a.meta = w.meta;
    L.bin_rows = w.bin_rows;
    L.rows = rows;
    L.giant_scratch = c.giant;
    L.giant_ctas = gctas;
    L.R_pad = R_pad;
    if (rows > 0) {
      SLG_TRY(launch_walk(L, st, &launches, evs.on ? evs.ev + kEvWalk : nullptr));
    } else if (evs.on) {
      for (int b = 0; b <= kNumBins; ++b) cudaEventRecord(evs.ev[kEvWalk + b], st);
    }
    SLG_TRY(launch_row_scan(rows, w, st));
    if (evs.on) cudaEventRecord(evs.ev[kEvScan], st);
    launches += 1 + 2 * (ntiles64 > 0);
    SLG_TRY(cudaMemcpyAsync(c.meta_host, w.meta, sizeof(Meta), cudaMemcpyDeviceToHost, st));
    SLG_TRY(cudaStreamSynchronize(st));
    const Meta &m = *c.meta_host;
    if (m.err) return m.err;
    pairs = (int64_t)m.pairs;
    if (op == kOpBuild) {
      if (pairs > capacity) {
        *result = pairs;
        return SLG_ERR_CAPACITY;
      }
      if (evs.on) cudaEventRecord(evs.ev[kEvGather0], st);
      if (pairs > 0) {
        if (m.stage_overflow == 0) {
          SLG_TRY(launch_gather(row_begin, rows, w, out_i, out_j, out_w, unweighted, st));
          launches += 1;
        } else {
          // Staging too small: walk again, writing straight to the output.
          SLG_TRY(cudaMemsetAsync(&w.meta->giant_ticket, 0, sizeof(unsigned int), st));
          L.a.mode = kDirect;
          L.a.row_ptr = w.row_ptr;
          L.a.out_i = out_i;
          L.a.out_j = out_j;
          L.a.out_w = out_w;
          SLG_TRY(launch_walk(L, st, &launches));
        }
        SLG_TRY(cudaMemcpyAsync(c.meta_host, w.meta, sizeof(Meta), cudaMemcpyDeviceToHost, st));
      }
      if (evs.on) cudaEventRecord(evs.ev[kEvGather1], st);
      SLG_TRY(cudaStreamSynchronize(st));
      if (c.meta_host->err) return c.meta_host->err;
    }
    *result = pairs;
  } else {
    SLG_TRY(cudaMemcpyAsync(c.meta_host, w.meta, sizeof(Meta), cudaMemcpyDeviceToHost, st));
    SLG_TRY(cudaStreamSynchronize(st));
    if (c.meta_host->err) return c.meta_host->err;
    *result = (int64_t)c.meta_host->wedges;
  }
  const Meta &m = *c.meta_host;
  stats.wedges = (int64_t)m.wedges;
  stats.pairs = pairs;
  stats.rows_active = (int64_t)m.active;
  for (int b = 0; b < kNumBins; ++b) {
    stats.rows_bin[b] = (int64_t)m.rows_bin[b];
    stats.wedges_bin[b] = (int64_t)m.wedges_bin[b];
    stats.incid_bin[b] = (int64_t)m.incid_bin[b];
    stats.pairs_bin[b] = (int64_t)m.pairs_bin[b];
  }
  stats.kernel_launches = launches;
  if (evs.on) {
    stats.profiled = 1;
    stats.ms_plan = evs.ms(kEvPlan, kEvWalk);
    for (int b = 0; b < kNumBins; ++b) stats.ms_walk[b] = evs.ms(kEvWalk + b, kEvWalk + b + 1);
    stats.ms_scan = evs.ms(kEvWalk + kNumBins, kEvScan);
    if (op == kOpBuild) stats.ms_gather = evs.ms(kEvGather0, kEvGather1);
  }
  t_stats = stats;
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
  int rc = check_args(hh, s, flags);
  if (rc != SLG_OK) return rc;
  if (!n_pairs || capacity < 0) return SLG_ERR_INVALID;
  const bool unweighted = (flags & SLG_UNWEIGHTED) != 0;
  if (capacity > 0 && (!out_i || !out_j || (!unweighted && !out_w))) return SLG_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  Pool pool(st);
  slg_hypergraph d = *hh;
  int32_t *e_off, *e_idx, *v_off, *v_idx, *oi = nullptr, *oj = nullptr, *ow = nullptr;
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
  d.e_off = e_off;
  d.e_idx = e_idx;
  d.v_off = v_off;
  d.v_idx = v_idx;
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
  SLG_TRY(cudaStreamSynchronize(st));
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
    default: return "unknown status";
  }
}

int slg_abi_version(void) { return SLG_ABI_VERSION; }

}  // extern "C"
