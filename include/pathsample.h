/*
 * pathsample.h -- C interface of the GPU path-sampling library.
 *
 * The library estimates the counts of all six connected induced 4-vertex
 * subgraphs of an undirected simple graph by 3-path sampling and centred
 * 3-path sampling (Jha, Seshadhri & Pinar, "Path Sampling: A Fast and
 * Provable Method for Estimating 4-Vertex Subgraph Counts").  Every step of
 * the sampling path runs in CUDA kernels for sm_103a (GB300).
 *
 * Motif numbering (the matrix of Eq. (1)): 1 = 3-star, 2 = 3-path,
 * 3 = tailed triangle, 4 = 4-cycle, 5 = chordal 4-cycle, 6 = 4-clique.
 *
 * Conventions for every call:
 *  - Pointers named d_* are device pointers; all others are host pointers.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *    queued on it; only the calls documented as synchronising wait for it.
 *  - The library never allocates device memory: all of it lives in the
 *    caller's workspace (see ps_graph_workspace_bytes).
 *  - Every call returns a status code (below); none throws, none traps the
 *    GPU.  Device-side faults in the input are reported through status codes.
 *  - Random draws are a pure function of (seed, sample id), so a range of
 *    sample ids gives the same class counts however it is split over calls,
 *    streams, launches or GPUs.
 */
#ifndef PATHSAMPLE_H
#define PATHSAMPLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *ps_stream_t; /* same type as cudaStream_t */

/* ---------------------------------------------------------------- status */
#define PS_OK 0
#define PS_NO_PATHS 1          /* W == 0 or Lambda == 0: nothing to sample      */
#define PS_ERR_ARG (-1)        /* bad argument, malformed offsets, column range */
#define PS_ERR_NOT_SIMPLE (-2) /* self-loop or repeated neighbour                */
#define PS_ERR_ASYMMETRIC (-3) /* an arc without its reverse                     */
#define PS_ERR_WORKSPACE (-4)  /* workspace missing, too small or misaligned     */
#define PS_ERR_OVERFLOW (-5)   /* W or Lambda does not fit in 64 bits            */
#define PS_ERR_TIMEOUT (-6)    /* a bounded device wait expired                  */
#define PS_ERR_CUDA (-7)       /* a CUDA runtime call failed                     */
#define PS_ERR_STATE (-8)      /* call out of order (e.g. sampling before prefix) */
#define PS_ERR_NOMEM (-9)      /* host allocation failed                         */
#define PS_ERR_TOO_LARGE (-10) /* input exceeds a fixed-size scratch limit        */

/* Tuning knobs.  None of them changes any result; they only change speed.
 * Pass NULL for the defaults; a zero field also means "default". */
typedef struct {
    int32_t block_size;         /* sampling threads per block: 128, 256 (default), 512, 1024 */
    int32_t blocks_per_sm;      /* resident sampling blocks per SM (default: occupancy)      */
    int32_t guide_log2_ratio;   /* guide buckets ~ m * 2^ratio, 1..4 (default 1, or m / 4
                                   buckets on graphs of 2^25 edges and more); -1 = none     */
    int32_t hub_count;          /* top-degree vertices (degree >= hub_min_degree) given an
                                   adjacency bitmap row; default: up to 1024 full-width
                                   rows within 256 MB (adjacency 2), up to 8192 rows of
                                   the hub span within 512 MB and 48 bytes per edge
                                   (adjacency 1, where a lookup whose larger label is a hub
                                   and whose smaller label is in the span reads its row);
                                   -1 = none                                                */
    int32_t samples_per_thread; /* samples each thread of the batched launch keeps in flight
                                   per step of its loop: 1 (default) or 2; the other
                                   samplers take one at a time                             */
    int32_t adjacency;          /* adjacency test: 1 = hash set of the edges (default),
                                   2 = search of the sorted smaller list + hub bitmaps,
                                   3 = a hash table per adjacency list                      */
    int32_t draw_order;         /* the *_ordered samplers: 0 (default) sort each chunk of
                                   samples by edge draw when the graph has >= 2^20 edges
                                   and the chunk >= 2^18 samples -- by 16 bits of r in two
                                   passes from 2^25 edges, by 8 bits below -- else take them
                                   in id order; 1 = always sort by 8 bits; 2 = always by
                                   16 bits; -1 = never                                      */
    int32_t hub_min_degree;     /* smallest degree given a hub bitmap row (default 64; the
                                   rows go to the top hub_count labels of at least this
                                   degree)                                                   */
    int32_t hub_span_log2;      /* hub rows hold the bits of the top 2^hub_span_log2 labels
                                   only (5..30; default 19 with adjacency 1, all labels
                                   with adjacency 2); -1 = all labels                       */
} ps_tuning;

/* Totals of one graph, filled by ps_tau_prefix. */
typedef struct {
    uint64_t W;       /* sum over edges of tau_e = (d_u - 1)(d_v - 1), Section 3       */
    uint64_t Lambda;  /* sum over edges of lambda_e = L_{u,v} L_{v,u}, Section 4        */
    uint64_t N1_lo;   /* N_1 = sum_v C(d_v, 3) (3-stars, Alg. 2) as a 128-bit integer  */
    uint64_t N1_hi;
    int64_t n;        /* vertices                                                        */
    int64_t m;        /* undirected edges                                                */
    int64_t d_max;    /* largest degree                                                  */
    int64_t hubs;     /* vertices with a bitmap row                                      */
    int32_t tau_shift;    /* guide bucket of r is r >> shift (tau prefix)               */
    int32_t lambda_shift; /* same for the lambda prefix                                  */
} ps_stats;

typedef struct ps_graph ps_graph; /* opaque; host metadata + pointers into the workspace */

/* Bytes of device workspace a graph with n vertices and nnz stored arcs
 * (nnz = 2m) needs under tuning t (NULL = defaults).  0 if the sizes are
 * outside the supported range (n < 2^31, nnz < 2^31).  Test hook: a
 * positive PS_TEST_ESET_LIST_CAP in the environment caps the hash set's
 * per-region key lists (forcing its overflow and slow paths; results are
 * unchanged); it must not change between this call and ps_load_csr. */
size_t ps_graph_workspace_bytes(int64_t n, int64_t nnz, const ps_tuning *t);

/* Section 2 input and Section 4 order.  Reads the CSR graph (d_off: int64
 * [n + 1], d_col: int32 [nnz]; rows in any order, both arc directions
 * stored), checks that it is an undirected simple graph, relabels every
 * vertex by its rank in the order "d_u < d_v, ties by smaller id" (so the
 * order becomes integer order), rebuilds the adjacency lists sorted
 * ascending, and builds the edge table (u < v, u ascending then v ascending)
 * with the positions of each edge in both endpoint lists, the inclusive
 * uint64 prefix sums of the weights tau_e and lambda_e (in the same pass as
 * the table), and (default adjacency) the hash set of the edges.
 *
 * d_off / d_col belong to the caller and are only read during the call.
 * d_workspace (ws_bytes >= ps_graph_workspace_bytes(n, nnz, t), 256-byte
 * aligned) must stay allocated and untouched until ps_graph_free(*out).
 * Synchronises `stream` (to read the validation flags).  The hash set build
 * (default adjacency), which only sampling reads, runs on a library-owned
 * stream and may still be running when the call returns: ps_tau_prefix
 * orders it before everything it queues on its own stream, and
 * ps_graph_free waits for it.  On error *out is NULL and the status is
 * PS_ERR_TIMEOUT (a bounded device wait of one of the scans expired, which
 * makes every other finding of the call unreliable, so it comes first) /
 * PS_ERR_ARG / PS_ERR_NOT_SIMPLE / PS_ERR_ASYMMETRIC (highest-priority
 * first) or PS_ERR_WORKSPACE / PS_ERR_CUDA. */
int ps_load_csr(int64_t n, int64_t nnz, const int64_t *d_off, const int32_t *d_col,
                void *d_workspace, size_t ws_bytes, const ps_tuning *t, ps_stream_t stream,
                ps_graph **out);

/* Section 3 (tau_e, W) and Section 4 (lambda_e, Lambda), the edge
 * distributions of Alg. 1 and Alg. 3: publishes the totals W and Lambda of
 * the inclusive uint64 prefix sums that ps_load_csr wrote (exact, so the edge
 * draw is exact), computes N_1 of Alg. 2, the guide tables of the
 * inverse-CDF search and the structures of the chosen adjacency variant; no
 * sampler may run before it.  Does not synchronise: the totals were read
 * back by ps_load_csr, *out is filled at once, and the guide tables and
 * adjacency structures are finished in `stream` order, so sampling on
 * another stream must first wait for `stream`.  A second call returns the same totals without
 * recomputing.  Returns PS_NO_PATHS when W == 0 or Lambda == 0
 * (sampling then leaves histograms untouched), PS_ERR_OVERFLOW when a sum
 * does not fit in 64 bits, PS_ERR_TIMEOUT when a scan's bounded wait
 * expired. */
int ps_tau_prefix(ps_graph *g, ps_stream_t stream, ps_stats *out);

/* Alg. 1 run k times, counted as in Alg. 2: sample ids first_id ..
 * first_id + k - 1, seed `seed`.  ADDS the class counts to d_hist6 (device,
 * uint64 [6]: triangle (u' == v', no motif), 3-path, tailed triangle,
 * 4-cycle, chordal 4-cycle, 4-clique).  Asynchronous on `stream`.  Returns
 * PS_NO_PATHS (and adds nothing) when W == 0. */
int ps_sample_3paths(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id,
                     uint64_t *d_hist6, ps_stream_t stream);

/* Alg. 3 run k times, counted as in Alg. 4.  ADDS to d_hist4 (device,
 * uint64 [4]: not centred, 4-cycle, chordal 4-cycle, 4-clique).
 * Asynchronous.  Returns PS_NO_PATHS (adds nothing) when Lambda == 0. */
int ps_sample_centered(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id,
                       uint64_t *d_hist4, ps_stream_t stream);

/* The same two samplers with the samples taken in the order of their edge
 * draws.  The samples of Alg. 1 and Alg. 3 are independent and the
 * histograms are sums, so the counts are exactly those of
 * ps_sample_3paths / ps_sample_centered for the same (k, seed, first_id);
 * only the memory traffic changes: the ids of each chunk are first sorted by
 * their draw r (256 or 65536 equal-width ranges of [0, W) or [0, Lambda);
 * see ps_tuning.draw_order), so samples in flight together read
 * neighbouring edge records and rows.
 *
 * d_scratch: caller-owned device memory, 16-byte aligned, of
 * ps_ordered_scratch_bytes(k_chunk) bytes (about 1 MB + 11 B per sample)
 * for chunks of k_chunk samples
 * (1 <= k_chunk <= 2^31; larger k runs in several chunks).  It is the
 * call's own working memory until the work queued on `stream` has run, so
 * concurrent calls need separate scratch.  Asynchronous.  Returns
 * PS_ERR_WORKSPACE when the scratch is missing, misaligned or smaller than
 * ps_ordered_scratch_bytes(1); otherwise as the plain samplers. */
size_t ps_ordered_scratch_bytes(uint64_t k_chunk);
int ps_sample_3paths_ordered(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id,
                             uint64_t *d_hist6, void *d_scratch, size_t scratch_bytes,
                             ps_stream_t stream);
int ps_sample_centered_ordered(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id,
                               uint64_t *d_hist4, void *d_scratch, size_t scratch_bytes,
                               ps_stream_t stream);

/* The estimators of Alg. 2 and Alg. 4 and the final combination of
 * Section 4 (C1..C3 from the 3-path counts, C4..C6 from the centred counts;
 * C1 = N_1 - C3 - 2 C5 - 4 C6 with the 3-path sampler's terms), plus the
 * error bars of Corollary 5.3 at confidence 1 - delta (the C1 bar adds those
 * of C3, 2 C5 and 4 C6).  Pure host function (FP64): hist6 / hist4 are host
 * copies of the histograms, k3 / kc their sample counts.  est, lo, hi
 * receive 6 values each, indexed by motif - 1.  Returns PS_ERR_ARG for
 * k3 == 0, kc == 0 or delta outside (0, 1); PS_NO_PATHS when W or Lambda is
 * 0 (the estimates are then exact: no 3-path / no 4-cycle exists). */
int ps_estimate(const ps_stats *st, const uint64_t hist6[6], uint64_t k3,
                const uint64_t hist4[4], uint64_t kc, double delta, double est[6],
                double lo[6], double hi[6]);

/* ps_estimate with options.  PS_EST_C1_FROM_CENTRED: C1 = N_1 - C3 - 2 C5 -
 * 4 C6 takes C5 and C6 (and their bars) from the centred sampler instead of
 * the 3-path sampler (C3 only the 3-path sampler sees).  The paper leaves
 * the choice open: Alg. 2 states the identity inside the 3-path algorithm,
 * while the end of Section 4 reports C4..C6 from the centred one.
 * PS_EST_3PATH_ONLY: report Alg. 2's own estimates of C4..C6 (3-path
 * sampler) instead of Alg. 4's, e.g. to compare the two samplers (Section 6);
 * hist4 and kc are then unused but must still be valid.  Unknown flag bits:
 * PS_ERR_ARG. */
#define PS_EST_C1_FROM_CENTRED 1u
#define PS_EST_3PATH_ONLY 2u
int ps_estimate_ex(const ps_stats *st, const uint64_t hist6[6], uint64_t k3,
                   const uint64_t hist4[4], uint64_t kc, double delta, uint32_t flags,
                   double est[6], double lo[6], double hi[6]);

/* Sampling until the error bars are narrow enough (the paper fixes k in
 * advance; this stops early from the same Corollary 5.3 bars).  Both samplers
 * draw ids [0, k) for k = k0, 2 k0, 4 k0, ... (capped at k_max, the last
 * look); after each look the estimates use confidence delta / L, L the number
 * of looks the schedule allows, so the union bound keeps the final bars at
 * confidence >= 1 - delta despite the early stop.  It stops at the first k
 * where every motif i (1..6) with bit i-1 of motif_mask set has
 * max(hi - est, est - lo) <= target * |est|, or at k_max.  d_hist6 /
 * d_hist4: device uint64 [6] / [4], zeroed by the call; the final
 * histograms equal one ps_sample_* call of k_used ids.  flags as in
 * ps_estimate_ex.  Synchronises `stream` after every look.  Returns
 * ps_estimate's status (PS_NO_PATHS stops after the first look). */
int ps_count_adaptive(const ps_graph *g, uint64_t seed, double target, double delta, uint64_t k0,
                      uint64_t k_max, uint32_t motif_mask, uint32_t flags, uint64_t *d_hist6,
                      uint64_t *d_hist4, ps_stream_t stream, uint64_t *k_used, uint64_t hist6[6],
                      uint64_t hist4[4], double est[6], double lo[6], double hi[6]);

/* Releases the host metadata of g (not the workspace, which the caller owns),
 * first waiting for library work that may still write into the workspace
 * (the hash set build of ps_load_csr); work the caller queued on its own
 * streams is the caller's to wait for. */
void ps_graph_free(ps_graph *g);

/* Short description of a status code (static string). */
const char *ps_strerror(int code);

/* Number of CUDA kernels this library has launched in this process so far
 * (all devices and threads).  For launch accounting in benchmarks. */
uint64_t ps_kernel_launches(void);

/* Self-test of failure detection: runs the bounded device wait that the
 * library's single-pass scans use, on a flag that nothing ever sets, and
 * returns the status the scans would report -- PS_ERR_TIMEOUT after
 * spin_limit polls (32-256 ns each; capped at the library's own limit)
 * instead of a hang.  d_scratch: device, 16 bytes, 16-byte aligned (cleared
 * by the call).  Synchronises `stream`; the context stays usable. */
int ps_selftest_bounded_wait(void *d_scratch, uint32_t spin_limit, ps_stream_t stream);

/* Which array ps_graph_copy copies out. */
#define PS_ARRAY_OFFSETS 0 /* int64 [n + 1]   canonical row offsets                      */
#define PS_ARRAY_COLUMNS 1 /* int32 [nnz]     canonical sorted adjacency                 */
#define PS_ARRAY_RANK 2    /* int32 [n]       canonical label of each input vertex       */
#define PS_ARRAY_EDGES 3   /* int32 [m][8]    u, v, d_u, d_v, iu, jv, off_u, off_v       */
#define PS_ARRAY_PTAU 4    /* uint64 [m]      inclusive prefix of tau                    */
#define PS_ARRAY_PLAMBDA 5 /* uint64 [m]      inclusive prefix of lambda                 */

/* Copies one device array of g into dst (host or device memory, `bytes` =
 * exactly the array's size) and synchronises `stream`.  For inspection and
 * tests. */
int ps_graph_copy(const ps_graph *g, int which, void *dst, size_t bytes, ps_stream_t stream);

/* ------------------------------------------------------------ end to end */

/* The whole path for one graph held in HOST memory (pinned for speed):
 * copies the CSR to the device, runs ps_load_csr, ps_tau_prefix, k3 3-path
 * and kc centred samples (seed, ids from 0), copies the histograms back and
 * fills est / lo / hi as ps_estimate.  hist6 / hist4 (host, may be NULL)
 * receive the class counts.  d_workspace must hold
 * ps_end_to_end_workspace_bytes(n, nnz, t) bytes; when it holds at least
 * ps_ordered_scratch_bytes(1) more, the rest is the scratch of the
 * draw-ordered samplers, which then take the samples (same counts).
 * Synchronises `stream`. */
size_t ps_end_to_end_workspace_bytes(int64_t n, int64_t nnz, const ps_tuning *t);
int ps_count_motifs_host(int64_t n, int64_t nnz, const int64_t *h_off, const int32_t *h_col,
                         uint64_t k3, uint64_t kc, uint64_t seed, double delta,
                         void *d_workspace, size_t ws_bytes, const ps_tuning *t,
                         ps_stream_t stream, uint64_t hist6[6], uint64_t hist4[4],
                         ps_stats *stats, double est[6], double lo[6], double hi[6]);

/* --------------------------------------------------------------- batched */

/* One unit of batched work: sample ids [first_id, first_id + count) of
 * graph `graph` (index into the table given to ps_batch_sample) with seed
 * `seed`, sampler 0 = Alg. 1 (adds into d_hist + 6 * slot), 1 = Alg. 3
 * (adds into d_hist + 6 * slot, first 4 words).  32 bytes. */
typedef struct {
    uint64_t first_id;
    uint64_t seed;
    uint32_t count;
    uint32_t graph;
    uint32_t slot;
    uint32_t sampler;
} ps_work;

/* Runs many work items, over many loaded graphs, in one persistent launch:
 * blocks take items from a device-side queue.  graphs: host array of
 * n_graphs handles (each after ps_tau_prefix); d_items: device array of
 * n_items ps_work; d_hist: device uint64 [6 * slots] (added to); d_table:
 * device scratch of ps_batch_table_bytes(n_graphs) bytes (graph descriptors,
 * written by this call); d_counter: device uint32 [2] (zeroed by this call;
 * afterwards [1] holds the number of items skipped because their graph's
 * adjacency variant differs from the one recorded for the table -- always 0
 * for tables written by ps_batch_prepare).  Each item's counts equal those of
 * the corresponding plain call.  When all graphs share one adjacency variant
 * the launch uses a kernel specialised for it.  Asynchronous. */
size_t ps_batch_table_bytes(int32_t n_graphs);
int ps_batch_sample(const ps_graph *const *graphs, int32_t n_graphs, const ps_work *d_items,
                    int64_t n_items, uint64_t *d_hist, void *d_table, uint32_t *d_counter,
                    const ps_tuning *t, ps_stream_t stream);

/* Writes the graph descriptors for ps_batch_sample_prepared into d_table
 * (d_table: device, ps_batch_table_bytes(n_graphs) bytes).  Synchronises
 * `stream`.  The graphs must stay loaded while the table is used. */
int ps_batch_prepare(const ps_graph *const *graphs, int32_t n_graphs, void *d_table,
                     ps_stream_t stream);
/* Same as ps_batch_sample with a table already written by ps_batch_prepare
 * (for capture in CUDA graphs: no host-to-device copy inside). */
int ps_batch_sample_prepared(const void *d_table, int32_t n_graphs, const ps_work *d_items,
                             int64_t n_items, uint64_t *d_hist, uint32_t *d_counter,
                             const ps_tuning *t, ps_stream_t stream);

/* ------------------------------------------------------ edge-list ingest */

/* Section 2's input from a raw edge list, on the device (the paper's
 * experiments start from edge lists, Section 6).  d_src / d_dst: device int32
 * [n_edges], edge i = {d_src[i], d_dst[i]}, ids in [0, n); either direction,
 * repeats and self-loops are allowed.  Writes the undirected simple graph:
 * self-loops dropped, both arcs of every remaining pair once, rows sorted
 * ascending -- d_off (device int64 [n + 1]) and d_col (device int32, room
 * for 2 n_edges entries; the first *nnz are written) -- ready for
 * ps_load_csr.  d_workspace: device, 256-byte aligned, at least
 * ps_ingest_workspace_bytes(n, n_edges) bytes (about 20 bytes per edge).
 * *nnz (host) receives the number of arcs.  Synchronises `stream`.  Returns
 * PS_ERR_ARG for an id outside [0, n) (or n, n_edges out of range: n < 2^31 - 1,
 * 2 n_edges < 2^31 - 1), PS_ERR_WORKSPACE for a missing, misaligned or small
 * workspace. */
size_t ps_ingest_workspace_bytes(int64_t n, int64_t n_edges);
int ps_csr_from_edges(int64_t n, int64_t n_edges, const int32_t *d_src, const int32_t *d_dst,
                      void *d_workspace, size_t ws_bytes, int64_t *d_off, int32_t *d_col,
                      int64_t *nnz, ps_stream_t stream);

/* ---------------------------------------------------------- exact counts */

/* Exact counts by enumeration, the ground truth that sampled estimates are
 * checked against where brute force is out of reach.  The paper obtains its
 * exact counts with separate enumeration code (Section 6) and does not
 * describe it; this call computes the non-induced counts N_1..N_6 of Eq. (1)
 * and inverts Eq. (1) for the induced counts C_1..C_6:
 *   N_1 = sum_v C(d_v, 3), N_2 = W - 3T (W counts each 3-path once and each
 *   triangle three times, Section 3), N_3 = sum over triangles of
 *   (d_a + d_b + d_c - 6), N_4 = 4-cycles, N_5 = sum over edges of
 *   C(t_e, 2) (t_e = triangles through e), N_6 = 4-cliques.
 * g must have been through ps_tau_prefix (it uses the canonical graph, W,
 * N_1 and g's adjacency test).  Work: one hash-set test per upper-part entry
 * of the lower endpoint of every edge, plus one per pair of common upper
 * neighbours (4-cliques), plus the wedges below each vertex (4-cycles).
 *
 * d_scratch: device, 256-byte aligned, at least
 * ps_exact_scratch_bytes(g, 1) bytes; ps_exact_scratch_bytes(g, 0) is the
 * size that lets the 4-cycle pass run on two blocks per SM (each block needs
 * 4 n bytes of counters).  On return its first 4 m bytes hold t_e (uint32,
 * edge order of PS_ARRAY_EDGES).  N (uint64 [6]) and C (int64 [6]) are host
 * arrays.  Synchronises `stream`.  Returns PS_ERR_STATE before
 * ps_tau_prefix, PS_ERR_WORKSPACE for a missing, misaligned or too small
 * scratch, PS_ERR_OVERFLOW when a count does not fit its type. */
size_t ps_exact_scratch_bytes(const ps_graph *g, int max_blocks);
int ps_count_exact(const ps_graph *g, void *d_scratch, size_t scratch_bytes, ps_stream_t stream,
                   uint64_t N[6], int64_t C[6]);

/* ------------------------------------------------------ allocation-free */

/* The paper has no counterpart to this call.  It is the exact prefix scan
 * that ps_tau_prefix runs over the tau / lambda weights, offered to callers
 * that cannot allocate device memory at all -- for example a plugin whose
 * host application owns every byte of device memory through its own pool,
 * or a serving process that reserved its whole HBM budget up front and must
 * not add allocations (or their implicit synchronisation) while requests are
 * in flight.  Such a caller can pass its own input and output buffers but no
 * workspace.
 *
 * Computes d_pa[i] = d_a[0] + ... + d_a[i] and d_pb[i] = d_b[0] + ... + d_b[i]
 * exactly in uint64 for i < count (device arrays; outputs may not alias the
 * inputs).  The scan's scratch is a fixed array of about 2.3 MB inside the
 * library that every GPU using the library keeps until the process exits;
 * the call allocates and frees no device memory and calls no allocating
 * library routine.  The first call on each device does the set-up: it looks
 * up that array's device address (with that device current; again after a
 * device reset, which gives the device a new context), and under CUDA's
 * default lazy loading that first call is also when the driver loads the
 * library's device code on the device and sets the array aside.  So make the
 * first call on each device at start-up, before requests are in flight and
 * before any stream capture.  All calls share the one array and it keeps the
 * last call's contents (each call clears what must start at zero), so calls
 * that overlap on the GPU (different streams or threads at once) race and
 * give wrong results; issue them one after another.  Synchronises `stream`.
 * Returns PS_ERR_TOO_LARGE (touching nothing) when count exceeds
 * PS_PREFIX_STATIC_MAX_ITEMS, PS_ERR_OVERFLOW when a sum does not fit in
 * 64 bits, PS_ERR_ARG for a negative count or a missing pointer. */
#define PS_PREFIX_STATIC_MAX_ITEMS (1ll << 27)
int ps_prefix_pairs_static(const uint64_t *d_a, const uint64_t *d_b, uint64_t *d_pa,
                           uint64_t *d_pb, int64_t count, ps_stream_t stream);

/* ------------------------------------------------------- measurement aid */

/* Not part of the method: reads the device buffer d_buf[0, bytes) `passes`
 * times with loads cached in L2 only (ld.global.cg), each block its own
 * even slice, and XORs a checksum into *d_sink (device, uint64) so the loads
 * stay.  Timing the call with events on `stream` gives, for a buffer that
 * fits in L2 (warm it with one pass first), the L2 read bandwidth that an
 * L2-resident graph's samplers are reported against.  Asynchronous.
 * PS_ERR_ARG when bytes is 0 or not a multiple of 16, d_buf is not 16-byte
 * aligned, passes <= 0 or a pointer is missing. */
int ps_l2_read_probe(const void *d_buf, uint64_t bytes, int32_t passes, uint64_t *d_sink,
                     ps_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* PATHSAMPLE_H */
