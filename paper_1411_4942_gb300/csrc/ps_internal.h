// ps_internal.h -- host-side internals shared by the library's translation
// units: the graph handle, the workspace layout and error helpers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pathsample.h"
#include "ps_device.cuh"
#include "ps_scan.cuh"

namespace ps {

// Sort tiers of the row relabel-and-sort step, by row length.
constexpr int kTierA = 32;      // one warp, one key per lane
constexpr int kTierB = 1024;    // one warp, up to 32 keys per lane in registers
constexpr int kTierC = 4096;    // one block, registers + 16 KB shared; above: block radix sort
// The edge hash set is built region by region in shared memory (64 KB of
// buckets each) once the table holds at least one whole region.
constexpr int64_t kRegionBuckets = 2048;
// Rows longer than this have their arcs walked by a whole block (lower-arc
// listing, hash set build); shorter rows by a warp per 32 rows.
constexpr int kLongRow = 128;
// Hub rows are only worth a bitmap above this degree (default of the tuning
// field hub_min_degree).
constexpr int kHubMinDegree = 64;
constexpr int kHubSpanLog2 = 19;   // default hub-row span beside the hash set
constexpr int kHubRowsMax = 8192;  // default hub-row cap beside the hash set
constexpr int64_t kCoarseGuideEdges = int64_t{1} << 25;  // default guide of m/4 buckets from here
// Items per tile of every scan.
constexpr int kScanBlock = 256;
constexpr int kScanItems = 8;
constexpr int64_t kScanTile = kScanBlock * kScanItems;
// Rank sort (LSD radix, 8-bit digits).
constexpr int kRadixBlock = 256;
constexpr int kRadixItems = 16;
constexpr int64_t kRadixTile = kRadixBlock * kRadixItems;

struct Tuning {
    int block_size;
    int blocks_per_sm;
    int guide_log2_ratio;  // >= 1: m << r buckets; -1: no guide; <= -2: m >> -r buckets
    int hub_count;         // 0: none
    int samples_per_thread;  // batched launch: 1 or 2
    int hub_min_degree;
    int hub_span_log2;     // hub rows cover the top 2^span labels; 0: all labels
    int adj_mode;          // kAdjHash or kAdjSearch
    int draw_order;        // ordered samplers: 0 by size, 1 always, -1 never
};
Tuning resolve_tuning(const ps_tuning *t, int64_t n, int64_t nnz);
// N_1 and the hub count into the status words (ps_prefix.cu); queued by the
// load step once the degrees are known
int launch_vertex_totals(ps_graph *g, cudaStream_t s);

struct Layout {
    int64_t n, nnz, m_cap, gcap, hub_cap, hub_words, hub_bit_base, radix_tiles, scan_tiles;
    int64_t eset_buckets;  // 0 without the edge hash set
    int64_t eset_regions;  // regions of the region build (0: the direct build)
    int64_t eset_cap, eset_ov_cap;  // region build: keys per region list, overflow list
    int64_t vtab_slots;    // 0 without the per-vertex tables
    size_t status, off, col, rank, lowcnt, ubase, dnew, rec, ptau, plam, gtau, glam, hub, eset, vtab;
    size_t keys0, keys1, vals0, vals1, rcounts, ecounts, ekeys, eregion, scan_flag, scan_agg, scan_inc;
    size_t total;
};
bool make_layout(int64_t n, int64_t nnz, const Tuning &t, Layout *L);

}  // namespace ps

struct ps_graph {
    ps::Layout L;
    ps::Tuning tune;
    char *ws;
    int device;
    int sm_count;
    int64_t n, nnz, m, d_max;
    // device arrays (inside ws)
    ps::u64 *status;
    int64_t *off;
    int32_t *col;
    int32_t *rank;
    int32_t *lowcnt;
    int64_t *ubase;
    int32_t *dnew;
    ps::EdgeRec *rec;
    uint64_t *ptau, *plam;
    int32_t *gtau, *glam;
    uint32_t *hub;
    uint64_t *eset;
    int32_t *vtab;
    bool prefixed;
    // read back at the end of ps_load_csr: W, Lambda, N_1 (lo, hi), the hub
    // count and the flags, so ps_tau_prefix needs no synchronisation
    uint64_t load_totals[5] = {0, 0, 0, 0, 0};
    uint64_t load_flags = 0;
    ps_stats stats;
    ps::GraphDev dev;
    // ev[0..2]: fork / join events of this graph's calls; ev[3]: end of the
    // edge hash set build, which runs on past ps_load_csr (eset_pending)
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    mutable bool eset_pending = false;
    ~ps_graph() {
        // the hash set build writes into the caller's workspace: let it end
        // (returns at once when it has, or was never started)
        if (ev[3]) cudaEventSynchronize(ev[3]);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
    }
};

namespace ps {

#define PS_CUDA_TRY(call)                         \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) return PS_ERR_CUDA; \
    } while (0)

int sm_count_of_current_device();
int flags_to_status(uint64_t flags);
// Two non-blocking streams of `device` for independent kernels within one
// call (created on first use, kept for the process; calls join them with
// their own events, so concurrent calls stay ordered correctly).
int get_side_streams(int device, cudaStream_t out[2]);

// Makes `s` wait for a hash set build still running from ps_load_csr; every
// call that reads the set (or the status words it writes) comes after this.
inline int wait_eset(const ps_graph *g, cudaStream_t s) {
    if (!g->eset_pending) return PS_OK;
    if (cudaStreamWaitEvent(s, g->ev[3], 0) != cudaSuccess) return PS_ERR_CUDA;
    g->eset_pending = false;
    return PS_OK;
}

// Every kernel launch is followed by this: counts the launch (reported by
// ps_kernel_launches) and checks the launch error.
void count_launch();
#define PS_LAUNCH_CHECK()                       \
    do {                                        \
        ::ps::count_launch();                   \
        PS_CUDA_TRY(cudaGetLastError());        \
    } while (0)

// Stable LSD radix-sort passes of ps_load.cu (8-bit digit at `shift`,
// uint32 keys with uint32 values, tiles of kRadixTile items): per-tile digit
// counts stored digit-major, then the scatter after their exclusive scan.
__global__ void __launch_bounds__(kRadixBlock)
k_radix_hist(int64_t n, const uint32_t *__restrict__ keys, int shift, uint32_t *counts, int64_t tiles);
__global__ void __launch_bounds__(kRadixBlock)
k_radix_scatter(int64_t n, const uint32_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                uint32_t *__restrict__ kout, uint32_t *__restrict__ vout, int shift,
                const uint32_t *__restrict__ offsets, int64_t tiles);

// scan helpers (ps_load.cu)
template <typename T>
ScanState<T> scan_state(ps_graph *g, int counter_slot);
int reset_scan(ps_graph *g, int counter_slot, int64_t count, cudaStream_t s);

// Scans `count` items of the graph's workspace through the shared scan
// state (one scan at a time per graph, in stream order).
template <typename T, typename Op, typename Load, typename Store>
inline int run_scan(ps_graph *g, int slot, int64_t count, T identity, Op op, Load load, Store store,
                    cudaStream_t s) {
    if (count <= 0) return PS_OK;
    int rc = reset_scan(g, slot, count, s);
    if (rc) return rc;
    const int64_t tiles = (count + kScanTile - 1) / kScanTile;
    k_scan<T, kScanBlock, kScanItems><<<(unsigned)tiles, kScanBlock, 0, s>>>(
        count, scan_state<T>(g, slot), identity, op, load, store);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

// The hash set's per-region key lists (region build): the edge-table
// kernel appends every edge's key to the list of its home bucket's region
// (cursors zeroed before); keys beyond a list's capacity go to an overflow
// list, and past that the slow path is flagged in status[ST_ESET_SPILL].
struct EsetLists {
    uint32_t *cur;       // [regions] list lengths
    uint32_t *ov_count;  // overflow list length
    uint64_t *keys;      // [regions][cap]
    uint64_t *ov_keys;   // [ov_cap]
    int64_t cap, ov_cap;
    uint64_t mask;       // buckets - 1
    int shift;           // region of bucket b = b >> shift
};

// The edge table (ps_edges.cu): after the rows are relabelled and sorted and
// ubase is known, writes every edge record (and, given `lists`, every edge's
// hash-set key into its region's list), and raises F_ASYM for an asymmetric
// input.
int build_edge_table(ps_graph *g, cudaStream_t s, const EsetLists *lists);
// Tiles of the edge table's radix sort for m edges (its digit counts take
// 256 words per tile).
int64_t edge_sort_tiles(int64_t m);

// steps (one translation unit each)
int load_graph(ps_graph *g, const int64_t *d_off, const int32_t *d_col, cudaStream_t s);
int prefix_graph(ps_graph *g, cudaStream_t s);
int launch_sampler(const ps_graph *g, int sampler, uint64_t k, uint64_t seed, uint64_t first_id,
                   uint64_t *d_hist, cudaStream_t s);
// Samples in the order of their edge draws (ps_order.cu); ids of a chunk are
// 32-bit offsets, so a chunk holds at most kOrderMaxChunk samples.
constexpr uint64_t kOrderMaxChunk = 1ull << 31;
size_t ordered_scratch_bytes(uint64_t k_chunk);
int launch_ordered(const ps_graph *g, int sampler, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *d_hist,
                   void *d_scratch, size_t scratch_bytes, cudaStream_t s);
int launch_batch(const void *d_table, int32_t n_graphs, const ps_work *d_items, int64_t n_items,
                 uint64_t *d_hist, uint32_t *d_counter, const Tuning &t, cudaStream_t s);
// Records the adjacency variant shared by a descriptor table's graphs (0: mixed).
void note_table_adjacency(const void *d_table, int adj);

}  // namespace ps
