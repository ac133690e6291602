/*
 * slg.h -- s-line graphs of hypergraphs on one GB300 (sm_103a): C ABI.
 *
 * The operation (Section III, definition of L_s(H)): H = (V, E) has
 * hyperedges e_0..e_{m-1}, each a set of vertices.  The weighted line graph
 * joins e_i and e_j (i != j) with weight w_ij = |e_i ∩ e_j| when the two
 * share a vertex; the s-line graph L_s(H) keeps the joins with w_ij >= s
 * (s >= 1).  The same construction on the dual H* (vertices and hyperedges
 * swapped, Section III) is selected with SLG_DUAL.
 *
 * Output format: the canonical edge list of L_s -- triples (i, j, w) with
 * i < j, w = |e_i ∩ e_j| >= s, listed in ascending (i, j) order, as three
 * int32 arrays (structure of arrays).  Ids are the caller's ids of the side
 * that was computed (hyperedge ids of H, or vertex ids of H for SLG_DUAL).
 * The result is unique and the library produces it bit for bit: every
 * count is an exact integer.
 *
 * Input format (Section III, the incidence of H and its bipartite form):
 * CSR (hyperedge -> vertices) and CSC (vertex -> hyperedges) of the same
 * incidence, int32 offsets and ids, every row strictly ascending, nnz < 2^31.
 *
 * Memory: unless stated otherwise, array arguments are DEVICE pointers on
 * the current CUDA device, owned by the caller, and are only read (inputs)
 * or written (outputs) during the call.  The library allocates its own
 * working memory from the device's stream-ordered pool and keeps a
 * zero-initialised scratch area per device between calls.  Calls are
 * enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and
 * return after one device->host read of the pair count, so *n_pairs and the
 * returned status are final on return; output arrays are complete once the
 * stream reaches that point (they are, since the call synchronises on it).
 *
 * Errors: every entry point returns an slg_status.  The library never
 * aborts the process and never traps the GPU: bad input detected on the
 * device is reported through a status word that the host reads.
 *
 * Thread safety: calls on different streams may run concurrently from
 * different host threads (their kernels overlap on the device); calls with
 * SLG_ALGO_PLAIN share a per-device scratch and are serialised.
 */
#ifndef SLG_H_
#define SLG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SLG_ABI_VERSION 8

/* Incidence of H as CSR + CSC (Section III: the hyperedge/vertex incidence
 * and its bipartite form).  All pointers are device pointers. */
typedef struct slg_hypergraph {
  int32_t n_edges;       /* m = |E|: rows of the CSR, >= 0 */
  int32_t n_vertices;    /* n = |V|: rows of the CSC, >= 0 */
  int64_t nnz;           /* number of incidences, 0 <= nnz < 2^31 */
  const int32_t *e_off;  /* [m+1] CSR offsets, e_off[0] = 0, e_off[m] = nnz */
  const int32_t *e_idx;  /* [nnz] vertex ids of each hyperedge, ascending */
  const int32_t *v_off;  /* [n+1] CSC offsets, v_off[0] = 0, v_off[n] = nnz */
  const int32_t *v_idx;  /* [nnz] hyperedge ids of each vertex, ascending */
} slg_hypergraph;

/* Status codes. */
typedef enum slg_status {
  SLG_OK = 0,
  SLG_ERR_INVALID = 1,     /* bad argument or malformed incidence */
  SLG_ERR_CAPACITY = 2,    /* output capacity < pair count; *n_pairs = count */
  SLG_ERR_NOMEM = 3,       /* device allocation failed */
  SLG_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  SLG_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  SLG_ERR_UNSUPPORTED = 6, /* flag combination not provided */
  SLG_ERR_TOO_LARGE = 7    /* input larger than slg_count_noalloc's fixed
                              working memory */
} slg_status;

/* Flags (bitwise OR). */
#define SLG_DUAL 0x1u        /* compute L_s(H*) instead of L_s(H) */
#define SLG_UNWEIGHTED 0x2u  /* stop counting a pair once it reaches s
                                (the short-circuit of Section IV-C); the
                                pair set is unchanged, out_w is not written
                                and may be NULL */
#define SLG_TENSOR_CORE 0x4u /* detect a dense core block of the incidence
                                and count its overlaps on the tensor cores
                                (slg_tile_overlap); the walk skips the core's
                                wedges and the tile counts are added before
                                the threshold, so the result is unchanged.
                                Binned algorithm only. */
#define SLG_RELABEL_ASC 0x8u  /* renumber the rows of the computed side by
                                ascending size before the walk (the
                                degree-ordered relabelling of Section IV-F),
                                then map the pairs back and restore the
                                canonical (i, j) order: the result is
                                unchanged, only which row carries each pair's
                                work differs.  Whole-side calls only (not
                                slg_build_rows, not plans); needs |L_s| <
                                2^31 for slg_build. */
#define SLG_RELABEL_DESC 0x10u /* the same by descending size; at most one
                                  of the two relabel flags */
#define SLG_NO_PRUNE 0x20u   /* switch off the degree-based pruning of
                                Algorithm 3 (rows of size < s stay in the
                                walk at both ends): same result, more work.
                                For ablations (Section V); binned algorithm
                                only */
#define SLG_ASYNC 0x40u      /* slg_build_host only: return once the copies
                                of the result to the host are enqueued on
                                `stream` (see slg_build_host) */
#define SLG_W16 0x80u        /* slg_build_host_many queries only: out_w is a
                                HOST uint16 array; the weights |e ∩ f| are
                                narrowed on the device before the copy back
                                (exact: a weight above 65,535 makes the
                                query fail with SLG_ERR_UNSUPPORTED) */
/* Algorithm selector (mutually exclusive values in bits 8..11). */
#define SLG_ALGO_MASK 0xF00u
#define SLG_ALGO_BINNED 0x000u /* default: degree-binned wedge walk */
#define SLG_ALGO_PLAIN 0x100u  /* plain per-hyperedge kernel: one warp per
                                  hyperedge, global count array (the
                                  paper's visited array), two passes */
#define SLG_ALGO_SPGEMM 0x200u /* filtered SpGEMM: both triangles of B·Bᵀ,
                                  no pruning, filter afterwards
                                  (Section IV-D) */

/*
 * slg_count -- number of pairs of L_s (Section III) without writing them.
 *   h        incidence of H (device arrays as described above)
 *   s        overlap threshold, s >= 1 (s larger than every hyperedge gives 0)
 *   flags    SLG_DUAL, SLG_UNWEIGHTED, SLG_TENSOR_CORE, SLG_RELABEL_ASC or
 *            SLG_RELABEL_DESC, SLG_NO_PRUNE, one SLG_ALGO_* value
 *   n_pairs  host pointer, receives |L_s|
 *   stream   cudaStream_t to run on
 * Returns SLG_OK, SLG_ERR_INVALID (s < 1, NULL pointers, negative sizes,
 * nnz >= 2^31, offsets not monotone, ids out of range, rows not strictly
 * ascending, CSR and CSC not the same incidence), SLG_ERR_NOMEM,
 * SLG_ERR_CUDA.
 */
int slg_count(const slg_hypergraph *h, int32_t s, uint32_t flags,
              int64_t *n_pairs, void *stream);

/*
 * slg_build -- the canonical edge list of L_s (Section III; Step 1 and
 * Step 2 of Section IV: s-overlaps, then the edge list).
 *   out_i, out_j, out_w  device int32 arrays of at least `capacity`
 *                        elements; out_w may be NULL with SLG_UNWEIGHTED
 *   capacity             elements available in each output array
 *   n_pairs              host pointer, receives |L_s|
 * When |L_s| > capacity the call returns SLG_ERR_CAPACITY with *n_pairs set
 * to the required count and the outputs unspecified.  Other errors as for
 * slg_count.
 */
int slg_build(const slg_hypergraph *h, int32_t s, uint32_t flags,
              int32_t *out_i, int32_t *out_j, int32_t *out_w,
              int64_t capacity, int64_t *n_pairs, void *stream);

/*
 * slg_build_rows -- rows [row_begin, row_end) of the canonical edge list
 * (the pairs whose smaller id i lies in the range), for streaming an output
 * that does not fit in memory at once.  Concatenating consecutive ranges
 * gives slg_build's result.  0 <= row_begin <= row_end <= rows of the side.
 */
int slg_build_rows(const slg_hypergraph *h, int32_t s, uint32_t flags,
                   int32_t row_begin, int32_t row_end, int32_t *out_i,
                   int32_t *out_j, int32_t *out_w, int64_t capacity,
                   int64_t *n_pairs, void *stream);

/*
 * slg_row_offsets -- where every row's pairs start in the canonical edge
 * list: row_ptr[r] = number of pairs (i, j) with i < r, row_ptr[R] = |L_s|
 * (one counting walk).  With it, an edge list too large for memory is
 * built in row ranges of bounded size with slg_build_rows.
 *   row_ptr  DEVICE int64 array of R + 1 entries (R = rows of the side)
 *   flags    SLG_DUAL, SLG_UNWEIGHTED, SLG_TENSOR_CORE, SLG_NO_PRUNE; binned
 *            algorithm only, no relabelling (SLG_ERR_UNSUPPORTED)
 * Synchronises `stream`.  Errors as for slg_count.
 */
int slg_row_offsets(const slg_hypergraph *h, int32_t s, uint32_t flags,
                    int64_t *row_ptr, void *stream);

/*
 * slg_build_host -- slg_build with every array in HOST memory: the call
 * copies the incidence to the device, builds L_s there and copies the
 * triples back (end-to-end use from host data).  `h` holds host pointers.
 * Pinned host memory makes the copies faster; pageable memory also works.
 * The input arrays may be reused when the call returns.  Without SLG_ASYNC
 * the call returns with out_i/out_j/out_w filled; with SLG_ASYNC it returns
 * (with *n_pairs set) once their device-to-host copies are enqueued on
 * `stream`: they are filled when the stream's work completes, so that calls
 * on different streams overlap one build's copies with the next one's walk.
 * Copy errors then surface when the stream is synchronised.
 */
int slg_build_host(const slg_hypergraph *h, int32_t s, uint32_t flags,
                   int32_t *out_i, int32_t *out_j, int32_t *out_w,
                   int64_t capacity, int64_t *n_pairs, void *stream);

/*
 * slg_build_csr -- slg_build's edge list in compressed row form: the pairs
 * of row i (the pairs (i, j) with i < j, ascending j) are
 * out_j[row_ptr[i] .. row_ptr[i + 1]) with their weights in out_w, so the
 * i of each pair is implied and not written.  This is L_s (Section III) as
 * the adjacency of its upper triangle; it moves a third fewer bytes than
 * the (i, j, w) triples.
 *   row_ptr  DEVICE int64 array of R + 1 entries (R = rows of the side);
 *            row_ptr[R] = |L_s|
 *   out_j, out_w, capacity, n_pairs  as for slg_build
 *   flags    as for slg_build except SLG_ALGO_SPGEMM and the relabel flags
 *            (SLG_ERR_UNSUPPORTED)
 * Synchronises `stream`.  Errors as for slg_build.
 */
int slg_build_csr(const slg_hypergraph *h, int32_t s, uint32_t flags,
                  int64_t *row_ptr, int32_t *out_j, int32_t *out_w,
                  int64_t capacity, int64_t *n_pairs, void *stream);

/*
 * One query of slg_build_host_many: L_s of the hypergraph or of its dual.
 *   s, flags   as for slg_build (SLG_ASYNC is not accepted), plus SLG_W16
 *              (out_w then points to uint16 host memory)
 *   row_ptr    HOST int64 array of R + 1 entries for the compressed row form
 *              of slg_build_csr (out_i unused, may be NULL), or NULL for the
 *              (i, j, w) triples of slg_build
 *   out_i, out_j, out_w, capacity   HOST arrays as for slg_build_host
 *   n_pairs    out: |L_s| (also when it exceeds capacity)
 *   status     out: this query's slg_status
 */
typedef struct slg_query {
  int32_t s;
  uint32_t flags;
  int64_t *row_ptr;
  int32_t *out_i, *out_j, *out_w;
  int64_t capacity;
  int64_t n_pairs;
  int32_t status;
} slg_query;

/*
 * slg_build_host_many -- several line graphs of one hypergraph given in
 * HOST memory (h holds host pointers): the incidence is copied to the
 * device once, the queries are built one after the other on `stream`, and
 * the result of each is copied back on a second stream of the call's own
 * while the next query is built.  Returns when every copy is done: SLG_OK
 * when every query succeeded, else the first failing query's status (each
 * query carries its own).  Pinned host arrays make the copies faster.
 */
int slg_build_host_many(const slg_hypergraph *h, slg_query *queries,
                        int32_t count, void *stream);

/*
 * slg_build_host_csr -- slg_build_host in the compressed row form of
 * slg_build_csr: row_ptr (HOST int64[R + 1]), out_j and out_w are host
 * arrays.  Synchronous.  Errors as for slg_build_csr.
 */
int slg_build_host_csr(const slg_hypergraph *h, int32_t s, uint32_t flags,
                       int64_t *row_ptr, int32_t *out_j, int32_t *out_w,
                       int64_t capacity, int64_t *n_pairs, void *stream);

/*
 * slg_row_work -- the wedge work of every row of the side: work[e] = number
 * of upper-triangle wedges e -> v -> f (|e|, |f| >= s) the walk visits for
 * row e (0 for rows of size < s); their sum is W_s (returned in *wedges).
 * Per-row work is what balances a split of the rows into contiguous ranges
 * for several GPUs (the parallel loop over hyperedges of Section IV-F).
 *   work    DEVICE int32 array of R entries (R = rows of the side)
 *   flags   SLG_DUAL, SLG_NO_PRUNE; binned algorithm only, no relabelling
 * Synchronises `stream`.  Errors as for slg_count.
 */
int slg_row_work(const slg_hypergraph *h, int32_t s, uint32_t flags,
                 int32_t *work, int64_t *wedges, void *stream);

/*
 * slg_wedges -- W_s, the number of upper-triangle wedges e -> v -> f
 * (f > e, |e| >= s, |f| >= s) that the walk visits: the exact work of the
 * s-overlap step after degree-based pruning (Section IV-C), equal to
 * sum over vertices of C(d_s(v), 2).  Device computation; host result.
 */
int slg_wedges(const slg_hypergraph *h, int32_t s, uint32_t flags,
               int64_t *wedges, void *stream);

/*
 * slg_filter -- L_s from the canonical edge list of L_s' for any s' <= s:
 * the triples with w >= s, in the same order (Section III: L_s keeps the
 * overlaps of weight >= s, so L_s ⊆ L_s' with equal weights).
 *   in_i, in_j, in_w     device arrays of n triples (a canonical edge list,
 *                        weighted); only read
 *   s                    threshold >= 1
 *   out_i, out_j, out_w  device arrays of `capacity` entries, not
 *                        overlapping the inputs; out_w may be NULL (weights
 *                        not written)
 *   n_pairs              host pointer, receives the kept count
 * Returns SLG_OK, SLG_ERR_INVALID, SLG_ERR_CAPACITY (*n_pairs = the kept
 * count, outputs unspecified), SLG_ERR_NOMEM, SLG_ERR_CUDA.
 */
int slg_filter(const int32_t *in_i, const int32_t *in_j, const int32_t *in_w,
               int64_t n, int32_t s, int32_t *out_i, int32_t *out_j,
               int32_t *out_w, int64_t capacity, int64_t *n_pairs,
               void *stream);

/*
 * slg_build_sweep -- L_s for `count` thresholds with one walk: L_{s_min}
 * (the smallest threshold) is built by slg_build, every other list is
 * filtered from it (slg_filter).
 *   s          HOST array of `count` thresholds (>= 1, any order), 1..64
 *   flags      as for slg_build except SLG_UNWEIGHTED (SLG_ERR_UNSUPPORTED:
 *              the weights decide membership)
 *   out_i, out_j, out_w   HOST arrays of `count` device pointers; list k
 *              receives L_{s[k]}.  out_w of the smallest threshold is
 *              required (the other lists are filtered by it); the others
 *              may be NULL
 *   capacity   HOST array of `count` capacities
 *   n_pairs    HOST array of `count` results; -1 where not computed
 * If the smallest threshold's list does not fit, returns SLG_ERR_CAPACITY
 * with only its count set.  If another list does not fit, every count is
 * set, the lists that fit are written, and SLG_ERR_CAPACITY is returned.
 * slg_last_stats describes the walk.  Other errors as for slg_build.
 */
int slg_build_sweep(const slg_hypergraph *h, const int32_t *s, int32_t count,
                    uint32_t flags, int32_t *const *out_i,
                    int32_t *const *out_j, int32_t *const *out_w,
                    const int64_t *capacity, int64_t *n_pairs, void *stream);

/*
 * After the edge list.  Inputs are device pair lists (i < j, ids in [0, R));
 * outputs are caller-owned device arrays.  Each call checks its input on
 * the device first (SLG_ERR_INVALID for an id out of range, i >= j, or --
 * where a canonical list is required -- pairs not strictly ascending) and
 * synchronises `stream` before it returns.
 *
 * slg_squeeze -- ID squeezing (Section IV-E): the ids that occur in the
 *   list are renumbered 0 .. n_ids-1 in ascending order of their original
 *   id (a canonical list stays canonical).
 *     out_i, out_j  [n] the list in new ids (may not overlap the input)
 *     old_of_new    [R] receives the original id of every new id (first
 *                   n_ids entries)
 *     n_ids         host pointer, receives the number of distinct ids
 *
 * slg_adjacency -- the adjacency of the line graph: symmetric CSR with V
 *   vertices built from a CANONICAL list (for instance a squeezed one, with
 *   V = n_ids).  Row v holds its neighbours in ascending order.
 *     adj_off  [V + 1] device int64 offsets
 *     adj      [2 n] neighbour ids; adj_w [2 n] their weights, or NULL
 *     in_w     required when adj_w is given
 *   n < 2^30.
 *
 * slg_components -- s-connected components: the connected components of
 *   L_s (Section I lists them as the analysis the s-line graph serves).
 *     labels        [R] receives for every id the smallest id of its
 *                   component (its own id when it occurs in no pair)
 *     n_components  host pointer, receives the number of components among
 *                   the ids that occur in the list
 *   R <= 2^24.  SLG_ERR_TIMEOUT if a bounded device loop gave up.
 */
int slg_squeeze(const int32_t *in_i, const int32_t *in_j, int64_t n, int32_t R,
                int32_t *out_i, int32_t *out_j, int32_t *old_of_new,
                int32_t *n_ids, void *stream);
int slg_adjacency(const int32_t *in_i, const int32_t *in_j, const int32_t *in_w,
                  int64_t n, int32_t V, int64_t *adj_off, int32_t *adj,
                  int32_t *adj_w, void *stream);
int slg_components(const int32_t *in_i, const int32_t *in_j, int64_t n,
                   int32_t R, int32_t *labels, int64_t *n_components,
                   void *stream);

/*
 * slg_tile_overlap -- exact overlap counts of a dense 0/1 block on the
 * tensor cores: C = A·Aᵀ, the linear-algebra form of Section IV-D applied to
 * a dense core of the incidence (the dense-core tile path).
 *   A          device bytes [rows_pad x cols_pad], row-major, 0x38 (FP8 E4M3
 *              1.0) for an incidence and 0x00 otherwise; 16-byte aligned
 *   rows_pad   multiple of 128;  cols_pad  multiple of 128, < 2^24
 *   C          device int32 [rows_pad x rows_pad], row-major; the tiles on
 *              and above the diagonal (128 x 128 blocks bj >= bi) receive
 *              C[i][j] = |row i ∩ row j| (exact: FP32 accumulation of 0/1
 *              products stays integral below 2^24); the others are untouched
 * Returns SLG_OK, SLG_ERR_INVALID (shape, alignment), SLG_ERR_UNSUPPORTED
 * (no tensor-map support in the driver), SLG_ERR_TIMEOUT (a bounded
 * device-side wait gave up), SLG_ERR_NOMEM, SLG_ERR_CUDA.
 */
int slg_tile_overlap(const uint8_t *A, int32_t rows_pad, int32_t cols_pad,
                     int32_t *C, void *stream);

/*
 * Batched form: many hypergraphs, each with its own threshold, built by one
 * pipeline.  The disjoint union of H_1 .. H_k has a block-diagonal incidence
 * (no vertex is shared), so every pair of its s-line graph lies inside one
 * member; with each row carrying its member's s_g the union's canonical edge
 * list is the members' lists, concatenated in member order (Section III
 * applied member by member).
 *
 * slg_plan_create -- builds the union on the device (copies of the members'
 *   arrays; the members may be freed afterwards), sizes every buffer with one
 *   counting pass, tunes the row-bin thresholds on this batch (a few timed
 *   builds) and captures the whole build into a CUDA graph.
 *     hs     HOST array of `count` hypergraphs whose arrays are device pointers
 *     s      HOST array of `count` thresholds (>= 1)
 *     flags  SLG_DUAL, SLG_UNWEIGHTED
 *     plan   receives the plan (free with slg_plan_destroy)
 *   Synchronises `stream`.  Errors as for slg_build; SLG_ERR_UNSUPPORTED for
 *   SLG_TENSOR_CORE, SLG_RELABEL_* or an algorithm flag.
 * slg_plan_execute -- replays the captured build on `stream`: one graph
 *   launch, no host synchronisation, results valid when the stream reaches
 *   that point.
 * slg_plan_result -- device pointers to the plan's output (owned by the plan;
 *   ids local to each member, pairs of member g at [offsets[g],
 *   offsets[g+1])); `offsets` is a HOST array of count + 1 entries (may be
 *   NULL); reads them synchronously.  Returns the device error status of the
 *   last execution, if any.
 * slg_plan_info -- the autotuner's choice, in `bins` (6 entries): the warp,
 *   CTA-small and CTA-large work limits, the sparse bin's upper work limit
 *   (0: bin off) and lower limit, and the dense-row ratio of the giant bin;
 *   the tuned build time in ms and the kernels per execution.
 */
typedef struct slg_plan slg_plan;
int slg_plan_create(const slg_hypergraph *hs, const int32_t *s, int32_t count,
                    uint32_t flags, slg_plan **plan, void *stream);
int slg_plan_execute(slg_plan *plan, void *stream);
int slg_plan_result(const slg_plan *plan, const int32_t **out_i,
                    const int32_t **out_j, const int32_t **out_w,
                    int64_t *n_pairs, int64_t *offsets);
int slg_plan_info(const slg_plan *plan, int32_t *bins, float *tuned_ms,
                  int32_t *launches);
int slg_plan_destroy(slg_plan *plan);

/*
 * slg_count_noalloc -- the same count as slg_count, for callers that must
 * not allocate device memory during the call.
 *
 * Who needs it: some callers cannot call cudaMalloc at the time they need
 * the count.  A process whose device memory is already claimed by another
 * allocator (for example a framework's caching allocator that reserves
 * nearly the whole GPU up front) would see the allocation fail.  A
 * latency-bound loop cannot afford an allocation that waits behind work
 * already queued on the device.  This entry point allocates nothing.  Its
 * working memory is one fixed 64 MiB device array built into the library,
 * which every GPU that loads the library keeps until the process exits.
 * The paper has no counterpart; this is a library convenience.
 *
 *   h, s, n_pairs, stream  as for slg_count
 *   flags                  SLG_DUAL and SLG_UNWEIGHTED only
 *
 * Limits and behaviour:
 *  - Size: the computed side may have at most 2,094,080 rows (hyperedges of
 *    H, or vertices with SLG_DUAL).  Larger inputs return SLG_ERR_TOO_LARGE
 *    without any device work.
 *  - The first call on a device looks up the array's device address (once
 *    per device); make that first call before any stream capture begins.
 *  - The call returns only once the count has reached the host: it waits
 *    for its stream.
 *  - Every call shares the array and keeps the previous call's contents.
 *    The result block is cleared at the start of every call; the counters
 *    and bitmaps are cleared too when the previous call on the device
 *    stopped with an error (a call that completes leaves them zero).  Calls
 *    whose work overlaps on the GPU (other streams, other host threads) race
 *    on the array: do not let them overlap.
 *  - The input is checked on the device as slg_count checks it: offsets, id
 *    ranges, strictly ascending rows and columns, and CSR and CSC describing
 *    the same incidence (SLG_ERR_INVALID otherwise).
 *  - It runs the plain per-hyperedge kernel (one warp per hyperedge), so it
 *    is slower than slg_count.
 */
int slg_count_noalloc(const slg_hypergraph *h, int32_t s, uint32_t flags,
                      int64_t *n_pairs, void *stream);

/* Statistics of the last call made by this host thread.  Bins: 0 = warp
 * (small rows), 1 = CTA small, 2 = CTA large, 3 = giant rows (dense in their
 * id span, s = 1, or dense-core rows), 4 = sparse large rows (s >= 2). */
typedef struct slg_stats {
  int64_t wedges;          /* W_s visited */
  int64_t pairs;           /* |L_s| */
  int64_t rows_active;     /* rows with size >= s */
  int64_t rows_bin[5];     /* rows per bin */
  int64_t wedges_bin[5];   /* wedges per bin */
  int64_t incid_bin[5];    /* CSR incidences of the rows of each bin */
  int64_t pairs_bin[5];    /* pairs emitted by each bin */
  int32_t kernel_launches; /* kernels launched by the call */
  int32_t profiled;        /* 1 if the ms_* fields below were measured */
  float ms_plan;           /* validation, maps, filtered CSC, bins */
  float ms_walk[5];        /* the walk kernel of each bin */
  float ms_scan;           /* row offsets */
  float ms_gather;         /* output assembly */
  int64_t core_rows;       /* dense core used by SLG_TENSOR_CORE: rows, */
  int64_t core_cols;       /* columns and incidences (0 when no core was */
  int64_t core_nnz;        /* found or the flag was not given) */
  int64_t giant_cycles[4]; /* giant bin, SM clock cycles summed over CTAs:
                              walk, partition into buckets, bucket counting
                              (of partitioned rows), and the whole of its
                              dense rows */
  int64_t max_row_work;    /* largest wedge count of one row */
  float ms_relabel;        /* SLG_RELABEL_*: building the renumbered side */
  float ms_order;          /* SLG_RELABEL_*: caller ids and (i, j) order */
  int64_t sparse_cycles[5]; /* sparse bin, SM clock cycles summed over CTAs:
                               row set-up, first walk, second pass (over the
                               copy of the far ends the first walk made),
                               collect and order the survivors, emit and
                               clear */
  float ms_tile;           /* the tensor-core tile kernel of the dense core
                              (SLG_TENSOR_CORE builds, slg_tile_overlap) */
} slg_stats;

int slg_last_stats(slg_stats *out);

/*
 * slg_set_core_params -- dense-core selection for SLG_TENSOR_CORE on later
 * calls from this host thread: candidate columns have degree >= tau_c and
 * candidate rows >= tau_r incidences in them; the columns are then re-taken
 * as those holding at least max(8, min_density x |rows|) candidate rows, and
 * the rows again against those columns.  The block is used when it has at
 * least 128 rows, 32 columns and a density >= min_density.
 * Defaults: 64, 32, 0.02.  Returns SLG_ERR_INVALID for values < 1 or a
 * density outside (0, 1].
 */
int slg_set_core_params(int32_t tau_c, int32_t tau_r, float min_density);

/*
 * slg_graph -- one device hypergraph prepared for several calls.  Every call
 * validates its input (offsets, id ranges, ascending rows and columns, CSR
 * and CSC the same incidence) and maps each CSR incidence to its CSC
 * position; a handle does both once, for both sides, and the builds and
 * counts made through it skip them.  The caller's arrays must stay valid and
 * unchanged while the handle lives.  Not a paper operation: a library
 * service for inputs that stay on the device (several thresholds or sides of
 * one hypergraph, served queries).
 * slg_graph_create -- validates h (errors as slg_count) and keeps 2 x nnz
 *   int32 of device memory for the maps; synchronises `stream`.
 * slg_graph_count, slg_graph_build -- slg_count and slg_build on the
 *   handle's hypergraph: the same arguments, flags, results and errors; a
 *   relabelling flag makes the call map its renumbered side itself.  Calls
 *   on one handle may run on several streams and host threads at once.
 *   SLG_ERR_INVALID when the current device is not the handle's.
 * slg_graph_destroy -- releases the handle's memory on the stream given to
 *   slg_graph_create (which must still exist) and waits for that stream.
 */
typedef struct slg_graph slg_graph;
int slg_graph_create(const slg_hypergraph *h, slg_graph **graph, void *stream);
int slg_graph_count(const slg_graph *graph, int32_t s, uint32_t flags, int64_t *n_pairs,
                    void *stream);
int slg_graph_build(const slg_graph *graph, int32_t s, uint32_t flags, int32_t *out_i,
                    int32_t *out_j, int32_t *out_w, int64_t capacity, int64_t *n_pairs,
                    void *stream);
int slg_graph_destroy(slg_graph *graph);

/* Returns the device memory that the library keeps for later calls on the
 * current device (its stream-ordered pool of working buffers) to the
 * system, after waiting for the device.  For processes where another
 * allocator (a framework's caching allocator) needs that memory.  Not a
 * paper operation: a library service. */
int slg_release_memory(void);

/* Per-phase CUDA-event timing of later calls from this host thread
 * (enable = 1) or not (0, the default).  Events are recorded on the call's
 * stream; the times land in slg_stats.ms_*. */
int slg_set_profiling(int enable);

/* Human-readable text for a status code (static storage). */
const char *slg_strerror(int status);

/* SLG_ABI_VERSION of the loaded library. */
int slg_abi_version(void);

/* Which device-side check raised the last error reported to this host
 * thread: 0 none, 1 row offsets, 2 row ids (range or order), 3 column
 * offsets, 4 column ids, 5 CSR and CSC differ, 6 a hash table or survivor
 * list exceeded its bound, 7 a giant-row scratch bound, 8 staged pairs
 * without staging room (a build that produced more pairs than counted). */
int slg_last_error_where(void);

#ifdef __cplusplus
}
#endif
#endif /* SLG_H_ */
