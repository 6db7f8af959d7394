// ps_api.cu -- the C entry points declared in include/pathsample.h: argument
// checks, workspace layout, the FP64 estimates and error bars, the
// end-to-end call and the batched-launch wrappers.
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ps_internal.h"

namespace ps {

namespace {

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Switches to the device that owns a graph for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

std::atomic<unsigned long long> g_launches{0};

}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

int sm_count_of_current_device() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return sms > 0 ? sms : 1;
}

int get_side_streams(int device, cudaStream_t out[2]) {
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static cudaStream_t streams[kMaxDevices][2] = {};
    if (device < 0 || device >= kMaxDevices) return PS_ERR_ARG;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < 2; ++i)
        if (!streams[device][i] && cudaStreamCreateWithFlags(&streams[device][i], cudaStreamNonBlocking) != cudaSuccess) {
            streams[device][i] = nullptr;
            return PS_ERR_CUDA;
        }
    out[0] = streams[device][0];
    out[1] = streams[device][1];
    return PS_OK;
}

// A scan whose bounded wait expired put identity in place of a predecessor's
// sum, so every later value of that call -- and any flag raised from them,
// such as a spurious overflow or asymmetry -- is unreliable: the timeout is
// reported first.
int flags_to_status(uint64_t f) {
    if (f & F_TIMEOUT) return PS_ERR_TIMEOUT;
    if (f & F_ARG) return PS_ERR_ARG;
    if (f & F_NOT_SIMPLE) return PS_ERR_NOT_SIMPLE;
    if (f & F_ASYM) return PS_ERR_ASYMMETRIC;
    if (f & F_OVERFLOW) return PS_ERR_OVERFLOW;
    return PS_OK;
}

Tuning resolve_tuning(const ps_tuning *t, int64_t n, int64_t nnz) {
    Tuning r;
    r.block_size = 256;
    r.blocks_per_sm = 0;
    // guide tables: 2m buckets; m/4 from kCoarseGuideEdges edges, where the
    // samplers take their draws in order (whole step on the 3M-vertex graph
    // 30.91 -> 29.76 ms with m/4, 30.38 with m, 30.01 with m/16 buckets;
    // R-MAT-20 4.32 ms either way)
    r.guide_log2_ratio = nnz / 2 >= kCoarseGuideEdges ? -2 : 1;
    r.samples_per_thread = 1;
    r.hub_min_degree = kHubMinDegree;
    r.adj_mode = kAdjHash;
    r.draw_order = 0;
    if (t && (t->adjacency == kAdjSearch || t->adjacency == kAdjVtab)) r.adj_mode = t->adjacency;
    // hub rows beside the hash set cover the top 2^19 labels only: a lookup
    // whose larger label is a hub and whose smaller is among them reads one
    // bit, the rest probe the set.  Narrower rows let more hubs share the
    // same bytes.  The search variant needs the rows for every hub pair and
    // keeps them full width.
    r.hub_span_log2 = r.adj_mode == kAdjHash ? kHubSpanLog2 : 0;
    if (t) {
        if (t->hub_span_log2 < 0) r.hub_span_log2 = 0;
        else if (t->hub_span_log2 > 0) r.hub_span_log2 = t->hub_span_log2 < 5 ? 5 : (t->hub_span_log2 > 30 ? 30 : t->hub_span_log2);
    }
    // hub bitmap rows: up to 1024 full-width rows within 256 MB for the search
    // variant; up to kHubRowsMax within 512 MB beside the hash set, and within
    // 48 bytes per edge there (under a third of the graph's workspace)
    const int64_t span = (r.hub_span_log2 > 0 && n > (int64_t{1} << r.hub_span_log2)) ? (int64_t{1} << r.hub_span_log2) : n;
    const int64_t row_bytes = ((span + 31) / 32) * 4;
    int64_t budget = (r.adj_mode == kAdjSearch ? 256ll : r.adj_mode == kAdjHash ? 512ll : 0ll) << 20;
    if (r.adj_mode == kAdjHash && budget > 24 * nnz) budget = 24 * nnz;
    int64_t hubs = row_bytes > 0 ? budget / row_bytes : 0;
    const int64_t cap = r.adj_mode == kAdjHash ? kHubRowsMax : 1024;
    if (hubs > cap) hubs = cap;
    r.hub_count = static_cast<int>(hubs);
    if (t) {
        if (t->block_size == 128 || t->block_size == 256 || t->block_size == 512 || t->block_size == 1024)
            r.block_size = t->block_size;
        if (t->blocks_per_sm > 0 && t->blocks_per_sm <= 32) r.blocks_per_sm = t->blocks_per_sm;
        if (t->guide_log2_ratio < 0) r.guide_log2_ratio = -1;
        else if (t->guide_log2_ratio > 0) r.guide_log2_ratio = t->guide_log2_ratio > 4 ? 4 : t->guide_log2_ratio;
        if (t->hub_count < 0) r.hub_count = 0;
        else if (t->hub_count > 0) r.hub_count = t->hub_count;
        if (t->samples_per_thread > 0) r.samples_per_thread = t->samples_per_thread >= 2 ? 2 : 1;
        if (t->hub_min_degree > 0) r.hub_min_degree = t->hub_min_degree;
        r.draw_order = t->draw_order >= 2 ? 2 : (t->draw_order > 0 ? 1 : (t->draw_order < 0 ? -1 : 0));
    }
    if (r.hub_count > n) r.hub_count = static_cast<int>(n);
    return r;
}

bool make_layout(int64_t n, int64_t nnz, const Tuning &t, Layout *L) {
    if (n < 0 || nnz < 0 || n >= INT32_MAX || nnz >= INT32_MAX) return false;
    Layout l{};
    l.n = n;
    l.nnz = nnz;
    l.m_cap = nnz / 2;
    // ratio r >= 1: m << r buckets; -1: none (at most 2 buckets); r <= -2
    // (the default on large graphs): m >> -r
    l.gcap = t.guide_log2_ratio == -1 ? 2
             : (t.guide_log2_ratio < 0 ? (l.m_cap >> -t.guide_log2_ratio) : (l.m_cap << t.guide_log2_ratio));
    if (l.gcap < 2) l.gcap = 2;
    if (l.gcap > INT32_MAX - 2) l.gcap = INT32_MAX - 2;  // bucket numbers stay in 31 bits
    l.hub_cap = t.hub_count;
    // hub rows hold the bits of the labels from hub_bit_base up (a multiple
    // of 32, at most the first hub's label)
    l.hub_bit_base = 0;
    if (t.hub_span_log2 > 0 && n > (int64_t{1} << t.hub_span_log2)) {
        int64_t base = n - (int64_t{1} << t.hub_span_log2);
        if (base > n - l.hub_cap) base = n - l.hub_cap;
        l.hub_bit_base = base > 0 ? (base / 32) * 32 : 0;
    }
    l.hub_words = (n - l.hub_bit_base + 31) / 32;
    // edge hash set: a power-of-two number of buckets, load <= 1/2
    l.eset_buckets = 0;
    if (t.adj_mode == kAdjHash) {
        int64_t slots = 64;
        while (slots < 2 * l.m_cap) slots <<= 1;
        l.eset_buckets = slots / kBucketSlots;
    }
    l.eset_regions = l.eset_buckets >= kRegionBuckets ? l.eset_buckets / kRegionBuckets : 0;
    // a region's keys are Poisson around m / regions (the hash is uniform), so
    // lists of 9/8 of that plus 64 overflow with negligible probability; the
    // overflow list catches the rest
    l.eset_cap = l.eset_regions ? (l.m_cap + l.eset_regions - 1) / l.eset_regions : 0;
    l.eset_cap += l.eset_cap / 8 + 64;
    l.eset_ov_cap = l.eset_regions ? 65536 + l.m_cap / 256 : 0;
    // test hook: PS_TEST_ESET_LIST_CAP=c caps every region list at c keys, so
    // the overflow list and, past it, the slow path take the other keys
    if (const char *cap_env = std::getenv("PS_TEST_ESET_LIST_CAP")) {
        const long long c = std::atoll(cap_env);
        if (l.eset_regions && c > 0 && c < l.eset_cap) l.eset_cap = c;
    }
    l.vtab_slots = t.adj_mode == kAdjVtab ? 2 * nnz : 0;
    l.radix_tiles = (n + kRadixTile - 1) / kRadixTile;
    if (l.radix_tiles < 1) l.radix_tiles = 1;
    int64_t scan_max = 256 * l.radix_tiles;
    if (n > scan_max) scan_max = n;
    if (l.m_cap > scan_max) scan_max = l.m_cap;
    if (l.gcap + 1 > scan_max) scan_max = l.gcap + 1;
    if (256 * edge_sort_tiles(l.m_cap) > scan_max) scan_max = 256 * edge_sort_tiles(l.m_cap);
    l.scan_tiles = (scan_max + kScanTile - 1) / kScanTile + 1;

    const size_t n1 = static_cast<size_t>(n > 0 ? n : 1);
    size_t p = 0;
    auto take = [&](size_t bytes) {
        const size_t at = p;
        p = align256(p + (bytes > 0 ? bytes : 1));
        return at;
    };
    l.status = take(ST_WORDS * sizeof(uint64_t));
    l.off = take((n1 + 1) * sizeof(int64_t));
    l.col = take(static_cast<size_t>(nnz) * sizeof(int32_t));
    l.rank = take(n1 * sizeof(int32_t));
    l.lowcnt = take(n1 * sizeof(int32_t));
    l.ubase = take((n1 + 1) * sizeof(int64_t));
    l.dnew = take(n1 * sizeof(int32_t));
    l.rec = take(static_cast<size_t>(l.m_cap) * sizeof(EdgeRec));
    l.ptau = take(static_cast<size_t>(l.m_cap) * sizeof(uint64_t));
    l.plam = take(static_cast<size_t>(l.m_cap) * sizeof(uint64_t));
    // G_tau also holds the edge sort's sorted (key, value) list during the load
    const int64_t gtau_words = l.gcap + 2 > 2 * l.m_cap ? l.gcap + 2 : 2 * l.m_cap;
    l.gtau = take(static_cast<size_t>(gtau_words) * sizeof(int32_t));
    l.glam = take(static_cast<size_t>(l.gcap + 2) * sizeof(int32_t));
    l.hub = take(static_cast<size_t>(l.hub_cap) * l.hub_words * sizeof(uint32_t));
    l.eset = take(static_cast<size_t>(l.eset_buckets) * kBucketSlots * sizeof(uint64_t));
    l.vtab = take(static_cast<size_t>(l.vtab_slots) * sizeof(int32_t));
    l.keys0 = take(n1 * sizeof(uint32_t));
    l.keys1 = take(n1 * sizeof(uint32_t));
    l.vals0 = take(n1 * sizeof(uint32_t));
    l.vals1 = take(n1 * sizeof(uint32_t));
    l.rcounts = take(static_cast<size_t>(256) * l.radix_tiles * sizeof(uint32_t));
    l.ecounts = take(static_cast<size_t>(256) * edge_sort_tiles(l.m_cap) * sizeof(uint32_t));
    // the region build's key lists (one per region, then the overflow list)
    // and their lengths
    l.ekeys = take(l.eset_regions ? static_cast<size_t>(l.eset_regions * l.eset_cap + l.eset_ov_cap) * sizeof(uint64_t)
                                  : 0);
    l.eregion = take(l.eset_regions ? static_cast<size_t>(l.eset_regions + 2) * sizeof(uint32_t) : 0);
    l.scan_flag = take(static_cast<size_t>(l.scan_tiles + 1) * sizeof(uint32_t));
    l.scan_agg = take(static_cast<size_t>(l.scan_tiles + 1) * sizeof(U64x2));
    l.scan_inc = take(static_cast<size_t>(l.scan_tiles + 1) * sizeof(U64x2));
    l.total = p;
    *L = l;
    return true;
}

// Corollary 5.3: p_l < alpha < p_u with exp(-k D(alpha, p)) = delta, D the
// Bernoulli KL divergence of Theorem 5.1; bisection on each side.
static double kl_div(double a, double b) {
    const double x = a > 0.0 ? a * std::log(a / b) : 0.0;
    const double y = a < 1.0 ? (1.0 - a) * std::log((1.0 - a) / (1.0 - b)) : 0.0;
    return x + y;
}

static void binomial_bar(uint64_t count, uint64_t k, double delta, double *pl, double *pu) {
    const double alpha = static_cast<double>(count) / static_cast<double>(k);
    const double target = std::log(1.0 / delta) / static_cast<double>(k);
    if (count == 0) {
        *pl = 0.0;
        *pu = 1.0 - std::pow(delta, 1.0 / static_cast<double>(k));
        return;
    }
    if (count == k) {
        *pl = std::pow(delta, 1.0 / static_cast<double>(k));
        *pu = 1.0;
        return;
    }
    // 200 halvings at most; once the midpoint rounds to an end the interval
    // can only stay or shrink onto that point, so stopping there returns the
    // same double as running on
    double a = 0.0, b = alpha;
    for (int i = 0; i < 200; i++) {
        const double mid = 0.5 * (a + b);
        if (mid == a || mid == b) break;
        if (kl_div(alpha, mid) > target) a = mid;
        else b = mid;
    }
    *pl = 0.5 * (a + b);
    a = alpha;
    b = 1.0;
    for (int i = 0; i < 200; i++) {
        const double mid = 0.5 * (a + b);
        if (mid == a || mid == b) break;
        if (kl_div(alpha, mid) > target) b = mid;
        else a = mid;
    }
    *pu = 0.5 * (a + b);
}

// Runs the bounded wait of the scans on a flag that nothing sets.
__global__ void k_wait_selftest(const uint32_t *flag, uint32_t limit, u64 *status) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && wait_flag(flag, limit) == 0u) raise_flag(status, F_TIMEOUT);
}

}  // namespace ps

using namespace ps;

extern "C" {

int ps_selftest_bounded_wait(void *d_scratch, uint32_t spin_limit, ps_stream_t stream) {
    if (!d_scratch || (reinterpret_cast<uintptr_t>(d_scratch) & 15u) != 0) return PS_ERR_ARG;
    if (spin_limit > kSpinLimit) spin_limit = kSpinLimit;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t *flag = static_cast<uint32_t *>(d_scratch);
    u64 *status = reinterpret_cast<u64 *>(static_cast<char *>(d_scratch) + 8);
    PS_CUDA_TRY(cudaMemsetAsync(d_scratch, 0, 16, s));
    k_wait_selftest<<<1, 32, 0, s>>>(flag, spin_limit, status - ST_FLAGS);
    PS_LAUNCH_CHECK();
    uint64_t flags = 0;
    PS_CUDA_TRY(cudaMemcpyAsync(&flags, status, sizeof(flags), cudaMemcpyDeviceToHost, s));
    PS_CUDA_TRY(cudaStreamSynchronize(s));
    return flags_to_status(flags);
}

size_t ps_graph_workspace_bytes(int64_t n, int64_t nnz, const ps_tuning *t) {
    Layout L;
    if (!make_layout(n, nnz, resolve_tuning(t, n, nnz), &L)) return 0;
    return L.total;
}

int ps_load_csr(int64_t n, int64_t nnz, const int64_t *d_off, const int32_t *d_col, void *d_workspace,
                size_t ws_bytes, const ps_tuning *t, ps_stream_t stream, ps_graph **out) {
    if (!out) return PS_ERR_ARG;
    *out = nullptr;
    if (n < 0 || nnz < 0 || !d_off || (nnz > 0 && !d_col)) return PS_ERR_ARG;
    const Tuning tu = resolve_tuning(t, n, nnz);
    Layout L;
    if (!make_layout(n, nnz, tu, &L)) return PS_ERR_ARG;
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) & 255u) != 0 || ws_bytes < L.total)
        return PS_ERR_WORKSPACE;
    ps_graph *g = new (std::nothrow) ps_graph();
    if (!g) return PS_ERR_NOMEM;
    g->L = L;
    g->tune = tu;
    g->ws = static_cast<char *>(d_workspace);
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return PS_ERR_CUDA;
    }
    g->sm_count = sm_count_of_current_device();
    for (cudaEvent_t &e : g->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            e = nullptr;
            delete g;
            return PS_ERR_CUDA;
        }
    g->n = n;
    g->nnz = nnz;
    char *ws = g->ws;
    g->status = reinterpret_cast<ps::u64 *>(ws + L.status);
    g->off = reinterpret_cast<int64_t *>(ws + L.off);
    g->col = reinterpret_cast<int32_t *>(ws + L.col);
    g->rank = reinterpret_cast<int32_t *>(ws + L.rank);
    g->lowcnt = reinterpret_cast<int32_t *>(ws + L.lowcnt);
    g->ubase = reinterpret_cast<int64_t *>(ws + L.ubase);
    g->dnew = reinterpret_cast<int32_t *>(ws + L.dnew);
    g->rec = reinterpret_cast<EdgeRec *>(ws + L.rec);
    g->ptau = reinterpret_cast<uint64_t *>(ws + L.ptau);
    g->plam = reinterpret_cast<uint64_t *>(ws + L.plam);
    g->gtau = reinterpret_cast<int32_t *>(ws + L.gtau);
    g->glam = reinterpret_cast<int32_t *>(ws + L.glam);
    g->hub = reinterpret_cast<uint32_t *>(ws + L.hub);
    g->eset = L.eset_buckets ? reinterpret_cast<uint64_t *>(ws + L.eset) : nullptr;
    g->vtab = L.vtab_slots ? reinterpret_cast<int32_t *>(ws + L.vtab) : nullptr;
    const int rc = load_graph(g, d_off, d_col, reinterpret_cast<cudaStream_t>(stream));
    if (rc != PS_OK) {
        delete g;
        return rc;
    }
    *out = g;
    return PS_OK;
}

int ps_tau_prefix(ps_graph *g, ps_stream_t stream, ps_stats *out) {
    if (!g) return PS_ERR_ARG;
    if (g->prefixed) {  // already done: the prefixes are in place
        if (out) *out = g->stats;
        return (g->stats.W == 0 || g->stats.Lambda == 0) ? PS_NO_PATHS : PS_OK;
    }
    DeviceGuard dg(g->device);
    if (!dg.ok) return PS_ERR_CUDA;
    const int rc = prefix_graph(g, reinterpret_cast<cudaStream_t>(stream));
    if ((rc == PS_OK || rc == PS_NO_PATHS) && out) *out = g->stats;
    return rc;
}

static int sample_common(const ps_graph *g, int sampler, uint64_t k, uint64_t seed, uint64_t first_id,
                         uint64_t *d_hist, ps_stream_t stream) {
    if (!g || !d_hist) return PS_ERR_ARG;
    if (!g->prefixed) return PS_ERR_STATE;
    const uint64_t total = sampler == 0 ? g->stats.W : g->stats.Lambda;
    if (total == 0) return PS_NO_PATHS;
    if (k == 0) return PS_OK;
    DeviceGuard dg(g->device);
    if (!dg.ok) return PS_ERR_CUDA;
    return launch_sampler(g, sampler, k, seed, first_id, d_hist, reinterpret_cast<cudaStream_t>(stream));
}

int ps_sample_3paths(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *d_hist6,
                     ps_stream_t stream) {
    return sample_common(g, 0, k, seed, first_id, d_hist6, stream);
}

int ps_sample_centered(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *d_hist4,
                       ps_stream_t stream) {
    return sample_common(g, 1, k, seed, first_id, d_hist4, stream);
}

size_t ps_ordered_scratch_bytes(uint64_t k_chunk) { return ordered_scratch_bytes(k_chunk); }

static int ordered_common(const ps_graph *g, int sampler, uint64_t k, uint64_t seed, uint64_t first_id,
                          uint64_t *d_hist, void *d_scratch, size_t scratch_bytes, ps_stream_t stream) {
    if (!g || !d_hist) return PS_ERR_ARG;
    if (!g->prefixed) return PS_ERR_STATE;
    if (!d_scratch || (reinterpret_cast<uintptr_t>(d_scratch) & 15u) != 0 ||
        scratch_bytes < ordered_scratch_bytes(1))
        return PS_ERR_WORKSPACE;
    const uint64_t total = sampler == 0 ? g->stats.W : g->stats.Lambda;
    if (total == 0) return PS_NO_PATHS;
    if (k == 0) return PS_OK;
    DeviceGuard dg(g->device);
    if (!dg.ok) return PS_ERR_CUDA;
    return launch_ordered(g, sampler, k, seed, first_id, d_hist, d_scratch, scratch_bytes,
                          reinterpret_cast<cudaStream_t>(stream));
}

int ps_sample_3paths_ordered(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *d_hist6,
                             void *d_scratch, size_t scratch_bytes, ps_stream_t stream) {
    return ordered_common(g, 0, k, seed, first_id, d_hist6, d_scratch, scratch_bytes, stream);
}

int ps_sample_centered_ordered(const ps_graph *g, uint64_t k, uint64_t seed, uint64_t first_id, uint64_t *d_hist4,
                               void *d_scratch, size_t scratch_bytes, ps_stream_t stream) {
    return ordered_common(g, 1, k, seed, first_id, d_hist4, d_scratch, scratch_bytes, stream);
}

int ps_estimate(const ps_stats *st, const uint64_t hist6[6], uint64_t k3, const uint64_t hist4[4],
                uint64_t kc, double delta, double est[6], double lo[6], double hi[6]) {
    return ps_estimate_ex(st, hist6, k3, hist4, kc, delta, 0u, est, lo, hi);
}

int ps_estimate_ex(const ps_stats *st, const uint64_t hist6[6], uint64_t k3, const uint64_t hist4[4],
                   uint64_t kc, double delta, uint32_t flags, double est[6], double lo[6], double hi[6]) {
    if (!st || !hist6 || !hist4 || !est || !lo || !hi) return PS_ERR_ARG;
    if (k3 == 0 || kc == 0 || !(delta > 0.0 && delta < 1.0)) return PS_ERR_ARG;
    if (flags & ~static_cast<uint32_t>(PS_EST_C1_FROM_CENTRED | PS_EST_3PATH_ONLY)) return PS_ERR_ARG;
    // 3-paths per motif (row 2 of Eq. (1)) and centred 3-paths (Lemma 4.2)
    static const double kA2[7] = {0, 0, 1, 2, 4, 6, 12};
    static const double kB[7] = {0, 0, 0, 0, 1, 1, 3};
    const unsigned __int128 n1w = (static_cast<unsigned __int128>(st->N1_hi) << 64) | st->N1_lo;
    const double n1 = static_cast<double>(n1w);
    // Alg. 2: every motif with a 3-path, from the 3-path sampler
    double c[7] = {0}, clo[7] = {0}, chi[7] = {0};
    if (st->W > 0) {
        for (int i = 2; i <= 6; i++) {
            c[i] = static_cast<double>(hist6[i - 1]) * static_cast<double>(st->W) / static_cast<double>(k3) / kA2[i];
            double pl, pu;
            binomial_bar(hist6[i - 1], k3, delta, &pl, &pu);
            const double scale = static_cast<double>(st->W) / kA2[i];
            clo[i] = pl * scale;
            chi[i] = pu * scale;
        }
    }
    // Alg. 4: the cycle-based motifs from the centred sampler
    double q[7] = {0}, qlo[7] = {0}, qhi[7] = {0};
    if (st->Lambda > 0) {
        for (int i = 4; i <= 6; i++) {
            q[i] = static_cast<double>(hist4[i - 3]) * static_cast<double>(st->Lambda) / static_cast<double>(kc) / kB[i];
            double pl, pu;
            binomial_bar(hist4[i - 3], kc, delta, &pl, &pu);
            const double scale = static_cast<double>(st->Lambda) / kB[i];
            qlo[i] = pl * scale;
            qhi[i] = pu * scale;
        }
    }
    // Alg. 2's induced 3-stars: N_1 - C_3 - 2 C_5 - 4 C_6, with C_5 and C_6 from
    // the 3-path sampler unless the flag asks for the centred ones (C_3 only
    // the 3-path sampler sees)
    const bool cen = (flags & PS_EST_C1_FROM_CENTRED) != 0;
    const double *e = cen ? q : c, *el = cen ? qlo : clo, *eh = cen ? qhi : chi;
    const double c1 = n1 - c[3] - 2.0 * e[5] - 4.0 * e[6];
    const double below = (c[3] - clo[3]) + 2.0 * (e[5] - el[5]) + 4.0 * (e[6] - el[6]);
    const double above = (chi[3] - c[3]) + 2.0 * (eh[5] - e[5]) + 4.0 * (eh[6] - e[6]);
    est[0] = c1;
    lo[0] = c1 - above;
    hi[0] = c1 + below;
    for (int i = 2; i <= 3; i++) {
        est[i - 1] = c[i];
        lo[i - 1] = clo[i];
        hi[i - 1] = chi[i];
    }
    // the final combination (end of Section 4): C_4..C_6 from Alg. 4, or on
    // request Alg. 2's own estimates of them
    const bool alg2 = (flags & PS_EST_3PATH_ONLY) != 0;
    for (int i = 4; i <= 6; i++) {
        est[i - 1] = alg2 ? c[i] : q[i];
        lo[i - 1] = alg2 ? clo[i] : qlo[i];
        hi[i - 1] = alg2 ? chi[i] : qhi[i];
    }
    return (st->W == 0 || st->Lambda == 0) ? PS_NO_PATHS : PS_OK;
}

// Looks of the doubling schedule k0, 2 k0, 4 k0, ..., capped at k_max.
static int adaptive_looks(uint64_t k0, uint64_t k_max) {
    int r = 1;
    for (uint64_t k = k0; k < k_max; k = (k > k_max / 2) ? k_max : 2 * k) r++;
    return r;
}

int ps_count_adaptive(const ps_graph *g, uint64_t seed, double target, double delta, uint64_t k0,
                      uint64_t k_max, uint32_t motif_mask, uint32_t flags, uint64_t *d_hist6,
                      uint64_t *d_hist4, ps_stream_t stream, uint64_t *k_used, uint64_t hist6[6],
                      uint64_t hist4[4], double est[6], double lo[6], double hi[6]) {
    if (!g || !d_hist6 || !d_hist4 || !k_used || !hist6 || !hist4 || !est || !lo || !hi) return PS_ERR_ARG;
    if (!g->prefixed) return PS_ERR_STATE;
    if (k0 == 0 || k_max < k0 || !(target > 0.0) || !(delta > 0.0 && delta < 1.0)) return PS_ERR_ARG;
    if ((motif_mask & ~0x3fu) != 0 ||
        (flags & ~static_cast<uint32_t>(PS_EST_C1_FROM_CENTRED | PS_EST_3PATH_ONLY)))
        return PS_ERR_ARG;
    DeviceGuard dg(g->device);
    if (!dg.ok) return PS_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    PS_CUDA_TRY(cudaMemsetAsync(d_hist6, 0, 6 * sizeof(uint64_t), s));
    PS_CUDA_TRY(cudaMemsetAsync(d_hist4, 0, 4 * sizeof(uint64_t), s));
    // the caller's confidence is split evenly over the looks (union bound)
    const double delta_look = delta / static_cast<double>(adaptive_looks(k0, k_max));
    uint64_t done = 0, k = k0;
    int rc = PS_OK;
    while (true) {
        const uint64_t add = k - done;
        if (g->stats.W > 0) rc = launch_sampler(g, 0, add, seed, done, d_hist6, s);
        if (rc == PS_OK && g->stats.Lambda > 0) rc = launch_sampler(g, 1, add, seed, done, d_hist4, s);
        if (rc != PS_OK) return rc;
        PS_CUDA_TRY(cudaMemcpyAsync(hist6, d_hist6, 6 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        PS_CUDA_TRY(cudaMemcpyAsync(hist4, d_hist4, 4 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
        PS_CUDA_TRY(cudaStreamSynchronize(s));
        done = k;
        rc = ps_estimate_ex(&g->stats, hist6, k, hist4, k, delta_look, flags, est, lo, hi);
        if (rc != PS_OK && rc != PS_NO_PATHS) return rc;
        bool met = true;
        for (int i = 0; i < 6; i++)
            if (motif_mask & (1u << i)) {
                const double half = std::fmax(hi[i] - est[i], est[i] - lo[i]);
                met = met && half <= target * std::fabs(est[i]);
            }
        if (met || rc == PS_NO_PATHS || k == k_max) break;
        k = (k > k_max / 2) ? k_max : 2 * k;
    }
    *k_used = done;
    return rc;
}

void ps_graph_free(ps_graph *g) { delete g; }

uint64_t ps_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char *ps_strerror(int code) {
    switch (code) {
        case PS_OK: return "ok";
        case PS_NO_PATHS: return "no 3-paths (W == 0) or no centred 3-paths (Lambda == 0)";
        case PS_ERR_ARG: return "invalid argument or malformed CSR";
        case PS_ERR_NOT_SIMPLE: return "graph has a self-loop or a repeated neighbour";
        case PS_ERR_ASYMMETRIC: return "graph is not symmetric (an arc lacks its reverse)";
        case PS_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case PS_ERR_OVERFLOW: return "W or Lambda does not fit in 64 bits";
        case PS_ERR_TIMEOUT: return "a bounded device wait expired";
        case PS_ERR_CUDA: return "CUDA runtime error";
        case PS_ERR_STATE: return "call out of order";
        case PS_ERR_NOMEM: return "host allocation failed";
        case PS_ERR_TOO_LARGE: return "input larger than the fixed scratch of an allocation-free call";
        default: return "unknown status";
    }
}

int ps_graph_copy(const ps_graph *g, int which, void *dst, size_t bytes, ps_stream_t stream) {
    if (!g || (!dst && bytes)) return PS_ERR_ARG;
    const void *src = nullptr;
    size_t want = 0;
    const size_t n = static_cast<size_t>(g->n), m = static_cast<size_t>(g->m);
    switch (which) {
        case PS_ARRAY_OFFSETS: src = g->off; want = (n + 1) * sizeof(int64_t); break;
        case PS_ARRAY_COLUMNS: src = g->col; want = static_cast<size_t>(g->nnz) * sizeof(int32_t); break;
        case PS_ARRAY_RANK: src = g->rank; want = n * sizeof(int32_t); break;
        case PS_ARRAY_EDGES: src = g->rec; want = m * sizeof(EdgeRec); break;
        case PS_ARRAY_PTAU: src = g->ptau; want = m * sizeof(uint64_t); break;
        case PS_ARRAY_PLAMBDA: src = g->plam; want = m * sizeof(uint64_t); break;
        default: return PS_ERR_ARG;
    }
    if ((which == PS_ARRAY_PTAU || which == PS_ARRAY_PLAMBDA) && !g->prefixed) return PS_ERR_STATE;
    if (bytes != want) return PS_ERR_ARG;
    if (want == 0) return PS_OK;
    DeviceGuard dg(g->device);
    if (!dg.ok) return PS_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    PS_CUDA_TRY(cudaMemcpyAsync(dst, src, want, cudaMemcpyDefault, s));
    PS_CUDA_TRY(cudaStreamSynchronize(s));
    return PS_OK;
}

// ------------------------------------------------------------- end to end

static size_t e2e_extra(int64_t n, int64_t nnz) {
    return align256(static_cast<size_t>(n + 1) * sizeof(int64_t)) +
           align256(static_cast<size_t>(nnz > 0 ? nnz : 1) * sizeof(int32_t)) + align256(16 * sizeof(uint64_t));
}

size_t ps_end_to_end_workspace_bytes(int64_t n, int64_t nnz, const ps_tuning *t) {
    const size_t g = ps_graph_workspace_bytes(n, nnz, t);
    return g ? g + e2e_extra(n, nnz) : 0;
}

int ps_count_motifs_host(int64_t n, int64_t nnz, const int64_t *h_off, const int32_t *h_col, uint64_t k3,
                         uint64_t kc, uint64_t seed, double delta, void *d_workspace, size_t ws_bytes,
                         const ps_tuning *t, ps_stream_t stream, uint64_t hist6[6], uint64_t hist4[4],
                         ps_stats *stats, double est[6], double lo[6], double hi[6]) {
    if (n < 0 || nnz < 0 || !h_off || (nnz > 0 && !h_col) || !est || !lo || !hi) return PS_ERR_ARG;
    const size_t gbytes = ps_graph_workspace_bytes(n, nnz, t);
    if (!gbytes) return PS_ERR_ARG;
    if (!d_workspace || ws_bytes < gbytes + e2e_extra(n, nnz)) return PS_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(d_workspace);
    int64_t *d_off = reinterpret_cast<int64_t *>(base + gbytes);
    int32_t *d_col = reinterpret_cast<int32_t *>(base + gbytes + align256(static_cast<size_t>(n + 1) * 8));
    uint64_t *d_hist = reinterpret_cast<uint64_t *>(reinterpret_cast<char *>(d_col) +
                                                    align256(static_cast<size_t>(nnz > 0 ? nnz : 1) * 4));
    PS_CUDA_TRY(cudaMemcpyAsync(d_off, h_off, static_cast<size_t>(n + 1) * sizeof(int64_t),
                                cudaMemcpyHostToDevice, s));
    if (nnz > 0)
        PS_CUDA_TRY(cudaMemcpyAsync(d_col, h_col, static_cast<size_t>(nnz) * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
    PS_CUDA_TRY(cudaMemsetAsync(d_hist, 0, 16 * sizeof(uint64_t), s));
    ps_graph *g = nullptr;
    int rc = ps_load_csr(n, nnz, d_off, d_col, d_workspace, gbytes, t, stream, &g);
    if (rc != PS_OK) return rc;
    ps_stats st{};
    rc = ps_tau_prefix(g, stream, &st);
    if (rc != PS_OK && rc != PS_NO_PATHS) {
        ps_graph_free(g);
        return rc;
    }
    // bytes beyond the minimum: scratch of the draw-ordered samplers
    const size_t used = gbytes + e2e_extra(n, nnz);
    void *oscr = static_cast<char *>(d_workspace) + used;
    const size_t obytes = ws_bytes - used;
    const bool ordered = obytes >= ordered_scratch_bytes(1);
    if (st.W > 0)
        rc = ordered ? ps_sample_3paths_ordered(g, k3, seed, 0, d_hist, oscr, obytes, stream)
                     : ps_sample_3paths(g, k3, seed, 0, d_hist, stream);
    if (rc >= 0 && st.Lambda > 0)
        rc = ordered ? ps_sample_centered_ordered(g, kc, seed, 0, d_hist + 8, oscr, obytes, stream)
                     : ps_sample_centered(g, kc, seed, 0, d_hist + 8, stream);
    if (rc < 0) {
        ps_graph_free(g);
        return rc;
    }
    uint64_t h[16];
    const cudaError_t e1 = cudaMemcpyAsync(h, d_hist, sizeof(h), cudaMemcpyDeviceToHost, s);
    const cudaError_t e2 = cudaStreamSynchronize(s);
    ps_graph_free(g);
    if (e1 != cudaSuccess || e2 != cudaSuccess) return PS_ERR_CUDA;
    if (hist6) std::memcpy(hist6, h, 6 * sizeof(uint64_t));
    if (hist4) std::memcpy(hist4, h + 8, 4 * sizeof(uint64_t));
    if (stats) *stats = st;
    return ps_estimate(&st, h, k3, h + 8, kc, delta, est, lo, hi);
}

// ---------------------------------------------------------------- batched

size_t ps_batch_table_bytes(int32_t n_graphs) {
    return n_graphs > 0 ? align256(static_cast<size_t>(n_graphs) * sizeof(GraphDev)) : 0;
}

int ps_batch_prepare(const ps_graph *const *graphs, int32_t n_graphs, void *d_table, ps_stream_t stream) {
    if (!graphs || n_graphs <= 0 || !d_table) return PS_ERR_ARG;
    std::vector<GraphDev> host(static_cast<size_t>(n_graphs));
    int adj = graphs[0] ? graphs[0]->dev.adj_mode : 0;
    for (int32_t i = 0; i < n_graphs; i++) {
        if (!graphs[i]) return PS_ERR_ARG;
        if (!graphs[i]->prefixed) return PS_ERR_STATE;
        host[static_cast<size_t>(i)] = graphs[i]->dev;
        if (graphs[i]->dev.adj_mode != adj) adj = 0;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    PS_CUDA_TRY(cudaMemcpyAsync(d_table, host.data(), host.size() * sizeof(GraphDev), cudaMemcpyHostToDevice, s));
    PS_CUDA_TRY(cudaStreamSynchronize(s));
    note_table_adjacency(d_table, adj);
    return PS_OK;
}

int ps_batch_sample_prepared(const void *d_table, int32_t n_graphs, const ps_work *d_items, int64_t n_items,
                             uint64_t *d_hist, uint32_t *d_counter, const ps_tuning *t, ps_stream_t stream) {
    if (!d_table || n_graphs <= 0 || n_items < 0 || (n_items > 0 && (!d_items || !d_hist)) || !d_counter)
        return PS_ERR_ARG;
    if (n_items > static_cast<int64_t>(UINT32_MAX) - (1 << 20)) return PS_ERR_ARG;
    const Tuning tu = resolve_tuning(t, 0, 0);
    return launch_batch(d_table, n_graphs, d_items, n_items, d_hist, d_counter, tu,
                        reinterpret_cast<cudaStream_t>(stream));
}

int ps_batch_sample(const ps_graph *const *graphs, int32_t n_graphs, const ps_work *d_items, int64_t n_items,
                    uint64_t *d_hist, void *d_table, uint32_t *d_counter, const ps_tuning *t,
                    ps_stream_t stream) {
    const int rc = ps_batch_prepare(graphs, n_graphs, d_table, stream);
    if (rc != PS_OK) return rc;
    return ps_batch_sample_prepared(d_table, n_graphs, d_items, n_items, d_hist, d_counter, t, stream);
}

}  // extern "C"
