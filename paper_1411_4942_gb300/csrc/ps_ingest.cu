// ps_ingest.cu -- ps_csr_from_edges: the undirected simple graph of Section 2
// from a raw edge list, on the device.  The paper's experiments read SNAP edge
// lists and time the whole run from them (Section 6); this turns such a list
// -- either direction, repeats, self-loops -- into the sorted symmetric CSR
// that ps_load_csr takes: self-loops dropped, both arcs of every remaining
// pair, each arc once, rows ascending.
//
// Both arcs of every edge go into (row, column) arrays; two stable radix
// sorts (by column, then by row) order them; the first copy of each arc is
// marked and its row counted; scans of the marks and of the row counts give
// each arc's position and the row offsets.
#include "ps_internal.h"

namespace ps {

namespace {

enum : int {
    IS_FLAGS = 0,     // F_ARG: an id outside [0, n)
    IS_NNZ = 1,       // arcs kept
    IS_COUNTER = 2,   // tile counters of the scans (one word each)
    IS_WORDS = 8,
};

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct IngestLayout {
    int64_t arcs, tiles, scan_tiles;
    size_t status, rows0, cols0, rows1, cols1, mark, deg, counts, scan_flag, scan_agg, scan_inc, total;
};

bool ingest_layout(int64_t n, int64_t n_edges, IngestLayout *L) {
    if (n < 0 || n >= INT32_MAX || n_edges < 0 || n_edges > (INT32_MAX - 1) / 2) return false;
    IngestLayout l{};
    l.arcs = 2 * n_edges;
    l.tiles = (l.arcs + kRadixTile - 1) / kRadixTile;
    if (l.tiles < 1) l.tiles = 1;
    int64_t scan_max = 256 * l.tiles;
    if (l.arcs > scan_max) scan_max = l.arcs;
    if (n > scan_max) scan_max = n;
    l.scan_tiles = (scan_max + kScanTile - 1) / kScanTile + 1;
    const size_t a = static_cast<size_t>(l.arcs > 0 ? l.arcs : 1);
    size_t p = 0;
    auto take = [&](size_t bytes) {
        const size_t at = p;
        p = align256(p + (bytes > 0 ? bytes : 1));
        return at;
    };
    l.status = take(IS_WORDS * sizeof(uint64_t));
    l.rows0 = take(a * sizeof(uint32_t));
    l.cols0 = take(a * sizeof(uint32_t));
    l.rows1 = take(a * sizeof(uint32_t));
    l.cols1 = take(a * sizeof(uint32_t));
    l.mark = take(a * sizeof(uint32_t));
    l.deg = take(static_cast<size_t>(n > 0 ? n : 1) * sizeof(int32_t));
    l.counts = take(static_cast<size_t>(256) * l.tiles * sizeof(uint32_t));
    l.scan_flag = take(static_cast<size_t>(l.scan_tiles + 1) * sizeof(uint32_t));
    l.scan_agg = take(static_cast<size_t>(l.scan_tiles + 1) * sizeof(int64_t));
    l.scan_inc = take(static_cast<size_t>(l.scan_tiles + 1) * sizeof(int64_t));
    l.total = p;
    *L = l;
    return true;
}

// Arc 2i = (u, v), arc 2i + 1 = (v, u) for edge i = (u, v); a self-loop
// becomes two copies of the sentinel (n, n), which sorts after every arc.
__global__ void k_ingest_arcs(int64_t n, int64_t n_edges, const int32_t *__restrict__ src,
                              const int32_t *__restrict__ dst, uint32_t *rows, uint32_t *cols,
                              u64 *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_edges; i += stride) {
        int32_t u = src[i], v = dst[i];
        if (u < 0 || u >= n || v < 0 || v >= n) {
            bad = true;
            u = v = static_cast<int32_t>(n);
        } else if (u == v) {
            u = v = static_cast<int32_t>(n);
        }
        rows[2 * i] = static_cast<uint32_t>(u);
        cols[2 * i] = static_cast<uint32_t>(v);
        rows[2 * i + 1] = static_cast<uint32_t>(v);
        cols[2 * i + 1] = static_cast<uint32_t>(u);
    }
    if (bad) raise_flag(status + IS_FLAGS, F_ARG);
}

// mark[i] = 1 for the first copy of each arc (the arcs are sorted by row,
// then column); deg[row] counts them.
__global__ void k_ingest_mark(int64_t n, int64_t arcs, const uint32_t *__restrict__ rows,
                              const uint32_t *__restrict__ cols, uint32_t *mark, int32_t *deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < arcs; i += stride) {
        const uint32_t r = rows[i], c = cols[i];
        const bool first = r < static_cast<uint64_t>(n) && (i == 0 || rows[i - 1] != r || cols[i - 1] != c);
        mark[i] = first ? 1u : 0u;
        if (first) atomicAdd(deg + r, 1);
    }
}

struct LoadMark {
    const uint32_t *mark;
    __device__ int64_t operator()(int64_t i) const { return mark[i]; }
};
// The kept arc i goes to position exc; the total is nnz.
struct StoreArcs {
    const uint32_t *cols;
    const uint32_t *mark;
    int32_t *col_out;
    u64 *status;
    int64_t arcs;
    __device__ void operator()(int64_t i, int64_t exc, int64_t inc) const {
        if (mark[i]) col_out[exc] = static_cast<int32_t>(cols[i]);
        if (i == arcs - 1) status[IS_NNZ] = static_cast<u64>(inc);
    }
};
struct LoadDegree {
    const int32_t *deg;
    __device__ int64_t operator()(int64_t i) const { return deg[i]; }
};
struct StoreRowOffsets {
    int64_t *off;
    int64_t n;
    __device__ void operator()(int64_t i, int64_t exc, int64_t inc) const {
        off[i] = exc;
        if (i == n - 1) off[n] = inc;
    }
};

template <typename T>
ScanState<T> ingest_scan_state(char *ws, const IngestLayout &L, int slot) {
    ScanState<T> s;
    s.flag = reinterpret_cast<uint32_t *>(ws + L.scan_flag);
    s.agg = reinterpret_cast<T *>(ws + L.scan_agg);
    s.inc = reinterpret_cast<T *>(ws + L.scan_inc);
    u64 *status = reinterpret_cast<u64 *>(ws + L.status);
    s.counter = reinterpret_cast<uint32_t *>(status + IS_COUNTER + slot);
    s.status = status + IS_FLAGS;
    return s;
}

template <typename T, typename Load, typename Store>
int ingest_scan(char *ws, const IngestLayout &L, int slot, int64_t count, T identity, Load load, Store store,
                cudaStream_t s) {
    if (count <= 0) return PS_OK;
    const int64_t tiles = (count + kScanTile - 1) / kScanTile;
    if (tiles > L.scan_tiles) return PS_ERR_WORKSPACE;
    PS_CUDA_TRY(cudaMemsetAsync(ws + L.scan_flag, 0, sizeof(uint32_t) * (tiles + 1), s));
    PS_CUDA_TRY(cudaMemsetAsync(reinterpret_cast<u64 *>(ws + L.status) + IS_COUNTER + slot, 0, sizeof(u64), s));
    k_scan<T, kScanBlock, kScanItems><<<(unsigned)tiles, kScanBlock, 0, s>>>(
        count, ingest_scan_state<T>(ws, L, slot), identity, OpSum(), load, store);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

struct LoadCount {
    const uint32_t *p;
    __device__ uint32_t operator()(int64_t i) const { return p[i]; }
};
struct StoreExclCount {
    uint32_t *p;
    __device__ void operator()(int64_t i, uint32_t exc, uint32_t) const { p[i] = exc; }
};

// Stable sort of `arcs` (key, value) pairs on the low `bits` bits of the key;
// returns with the sorted pairs in (*k, *v), the other pair of buffers scratch.
int ingest_sort(char *ws, const IngestLayout &L, int64_t arcs, int bits, uint32_t **k, uint32_t **v,
                uint32_t **k_alt, uint32_t **v_alt, int slot, cudaStream_t s) {
    uint32_t *counts = reinterpret_cast<uint32_t *>(ws + L.counts);
    const int64_t tiles = (arcs + kRadixTile - 1) / kRadixTile;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<<<(unsigned)tiles, kRadixBlock, 0, s>>>(arcs, *k, shift, counts, tiles);
        PS_LAUNCH_CHECK();
        int rc = ingest_scan<uint32_t>(ws, L, slot, 256 * tiles, 0u, LoadCount{counts}, StoreExclCount{counts}, s);
        if (rc) return rc;
        k_radix_scatter<<<(unsigned)tiles, kRadixBlock, 0, s>>>(arcs, *k, *v, *k_alt, *v_alt, shift, counts, tiles);
        PS_LAUNCH_CHECK();
        uint32_t *t = *k;
        *k = *k_alt;
        *k_alt = t;
        t = *v;
        *v = *v_alt;
        *v_alt = t;
    }
    return PS_OK;
}

}  // namespace

}  // namespace ps

using namespace ps;

extern "C" size_t ps_ingest_workspace_bytes(int64_t n, int64_t n_edges) {
    IngestLayout L;
    return ingest_layout(n, n_edges, &L) ? L.total : 0;
}

extern "C" int ps_csr_from_edges(int64_t n, int64_t n_edges, const int32_t *d_src, const int32_t *d_dst,
                                 void *d_workspace, size_t ws_bytes, int64_t *d_off, int32_t *d_col,
                                 int64_t *nnz, ps_stream_t stream) {
    if (!nnz || !d_off || n_edges < 0 || (n_edges > 0 && (!d_src || !d_dst || !d_col))) return PS_ERR_ARG;
    *nnz = 0;
    IngestLayout L;
    if (!ingest_layout(n, n_edges, &L)) return PS_ERR_ARG;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u) != 0 || ws_bytes < L.total)
        return PS_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(d_workspace);
    u64 *status = reinterpret_cast<u64 *>(ws + L.status);
    int32_t *deg = reinterpret_cast<int32_t *>(ws + L.deg);
    uint32_t *rows = reinterpret_cast<uint32_t *>(ws + L.rows0);
    uint32_t *cols = reinterpret_cast<uint32_t *>(ws + L.cols0);
    uint32_t *rows_alt = reinterpret_cast<uint32_t *>(ws + L.rows1);
    uint32_t *cols_alt = reinterpret_cast<uint32_t *>(ws + L.cols1);
    uint32_t *mark = reinterpret_cast<uint32_t *>(ws + L.mark);
    const int sms = sm_count_of_current_device();
    PS_CUDA_TRY(cudaMemsetAsync(status, 0, IS_WORDS * sizeof(u64), s));
    PS_CUDA_TRY(cudaMemsetAsync(deg, 0, static_cast<size_t>(n > 0 ? n : 1) * sizeof(int32_t), s));
    if (L.arcs > 0) {
        k_ingest_arcs<<<sms * 8, 256, 0, s>>>(n, n_edges, d_src, d_dst, rows, cols, status);
        PS_LAUNCH_CHECK();
        // ids and the sentinel are <= n: sort on the bits of n
        int bits = 1;
        while (bits < 32 && (static_cast<uint64_t>(n) >> bits) != 0) bits++;
        // by column, then (stably) by row: (row, column) order
        int rc = ingest_sort(ws, L, L.arcs, bits, &cols, &rows, &cols_alt, &rows_alt, 0, s);
        if (rc) return rc;
        rc = ingest_sort(ws, L, L.arcs, bits, &rows, &cols, &rows_alt, &cols_alt, 0, s);
        if (rc) return rc;
        k_ingest_mark<<<sms * 8, 256, 0, s>>>(n, L.arcs, rows, cols, mark, deg);
        PS_LAUNCH_CHECK();
        rc = ingest_scan<int64_t>(ws, L, 1, L.arcs, (int64_t)0, LoadMark{mark},
                                  StoreArcs{cols, mark, d_col, status, L.arcs}, s);
        if (rc) return rc;
    }
    PS_CUDA_TRY(cudaMemsetAsync(d_off, 0, sizeof(int64_t), s));
    int rc = ingest_scan<int64_t>(ws, L, 2, n, (int64_t)0, LoadDegree{deg}, StoreRowOffsets{d_off, n}, s);
    if (rc) return rc;
    uint64_t st[IS_WORDS];
    PS_CUDA_TRY(cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, s));
    PS_CUDA_TRY(cudaStreamSynchronize(s));
    const int status_code = flags_to_status(st[IS_FLAGS]);
    if (status_code != PS_OK) return status_code;
    *nnz = static_cast<int64_t>(st[IS_NNZ]);
    return PS_OK;
}
