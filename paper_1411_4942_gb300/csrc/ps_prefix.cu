// ps_prefix.cu -- ps_tau_prefix: the edge weights of Section 3 (tau) and
// Section 4 (lambda), their exact inclusive uint64 prefixes (the
// distributions p_e of Alg. 1 / Alg. 3), N_1 of Alg. 2, the guide
// tables that shorten the inverse-CDF search, and the hub bitmaps used by
// the adjacency test.
#include "ps_internal.h"

namespace ps {

// N_1 = sum_v C(d_v, 3) (128-bit) and the number of hub rows: the top
// `hub_cap` labels whose degree is at least `hub_min` (labels are in degree
// order, so these are the last rows).
__global__ void __launch_bounds__(256)
k_vertex_totals(int64_t n, const int32_t *__restrict__ dnew, int64_t hub_cap, int64_t hub_min, u64 *status) {
    uint64_t lo = 0, hi = 0;
    unsigned long long hubs = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const uint64_t d = static_cast<uint64_t>(dnew[r]);
        if (d >= 3) {
            // d (d - 1) (d - 2) / 6 with d < 2^31: the product fits in 128 bits
            const uint64_t a = d * (d - 1);  // < 2^62
            const uint64_t b = d - 2;
            uint64_t plo = a * b, phi = __umul64hi(a, b);
            // divide the 128-bit product by 6 (exact)
            const uint64_t qhi = phi / 6, rhi = phi % 6;
            // (rhi * 2^64 + plo) / 6 with rhi < 6
            const unsigned __int128 rest = (static_cast<unsigned __int128>(rhi) << 64) | plo;
            const uint64_t qlo = static_cast<uint64_t>(rest / 6);
            add128(lo, hi, qlo);
            hi += qhi;
        }
        if (r >= n - hub_cap && d >= static_cast<uint64_t>(hub_min)) hubs++;
    }
    warp_add128(lo, hi);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hubs += __shfl_down_sync(0xffffffffu, hubs, o);
    if ((threadIdx.x & 31) == 0) {
        if (lo | hi) atomic_add128(status + ST_N1_LO, lo, hi);
        if (hubs) atomicAdd(reinterpret_cast<unsigned long long *>(status + ST_HUBS), hubs);
    }
}

// Guide table: bucket b holds r in [b << shift, (b + 1) << shift), and G[b]
// is the edge that the first r of bucket b selects.  Edge j covers r in
// [P[j-1], P[j] - 1], so it owns the buckets whose first r falls in that
// range -- a contiguous run, and every bucket has exactly one owner.  Each
// lane writes its own short run; a warp writes long runs together.  A warp
// takes kGuideGroups groups of 32 edges per step with all their prefix loads
// issued first.
constexpr int kGuideGroups = 4;

__global__ void __launch_bounds__(256)
k_guide_fill(int64_t m, const uint64_t *__restrict__ P, int shift, int32_t *G, int64_t B) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * blockDim.x / 32;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (blockIdx.x == 0 && threadIdx.x == 0) G[B] = static_cast<int32_t>(m - 1);
    for (int64_t g0 = wid * kGuideGroups; g0 * 32 < m; g0 += nw * kGuideGroups) {
        uint64_t prev[kGuideGroups], cur[kGuideGroups];
#pragma unroll
        for (int u = 0; u < kGuideGroups; u++) {
            const int64_t j = (g0 + u) * 32 + lane;
            prev[u] = (j >= 1 && j <= m) ? __ldg(P + j - 1) : 0ull;
            cur[u] = j < m ? __ldg(P + j) : 0ull;
        }
        // bucket numbers are below B + 1 <= 2^31, so after the shift the runs
        // are handled in 32 bits
#pragma unroll
        for (int u = 0; u < kGuideGroups; u++) {
            const int64_t j = (g0 + u) * 32 + lane;
            uint32_t bstart = 0, len = 0;
            if (j < m && cur[u] != prev[u]) {
                bstart = prev[u] ? static_cast<uint32_t>((prev[u] - 1) >> shift) + 1u : 0u;
                const uint32_t bend = static_cast<uint32_t>((cur[u] - 1) >> shift);
                len = bstart <= bend ? bend - bstart + 1u : 0u;
            }
            if (len <= 8) {
                for (uint32_t q = 0; q < len; q++) G[bstart + q] = static_cast<int32_t>(j);
            }
            uint32_t longs = __ballot_sync(0xffffffffu, len > 8);
            while (longs) {
                const int l = __ffs(longs) - 1;
                longs &= longs - 1;
                const uint32_t bs = __shfl_sync(0xffffffffu, bstart, l);
                const uint32_t ln = __shfl_sync(0xffffffffu, len, l);
                const int32_t jj = static_cast<int32_t>((g0 + u) * 32 + l);
                for (uint32_t q = lane; q < ln; q += 32) G[bs + q] = jj;
            }
        }
    }
}

// Hub bitmap rows, one block per (hub, chunk of 2^20 labels): the block sets
// bit x for every neighbour x inside its chunk in shared memory, then writes
// the chunk out whole (coalesced), so no clearing pass and no global atomics.
constexpr int kHubThreads = 1024;
constexpr int64_t kHubChunkWords = 1 << 15;  // 128 KB of shared memory

__global__ void __launch_bounds__(kHubThreads)
k_hub_rows(int64_t hub_start, int64_t bit_base, const int64_t *__restrict__ coff, const int32_t *__restrict__ ccol,
           uint32_t *bits, int64_t words, int64_t chunks) {
    extern __shared__ uint32_t s_row[];
    const int64_t h = blockIdx.x / chunks, c = blockIdx.x % chunks;
    const int64_t w0 = c * kHubChunkWords;
    const int64_t nw = min(kHubChunkWords, words - w0);
    for (int64_t w = threadIdx.x; w < nw; w += kHubThreads) s_row[w] = 0u;
    __syncthreads();
    const int64_t r = hub_start + h;
    const int64_t o = coff[r], e = coff[r + 1];
    const int64_t lo = bit_base + w0 * 32, hi = bit_base + (w0 + nw) * 32;  // bit_base % 32 == 0
    for (int64_t i = o + threadIdx.x; i < e; i += kHubThreads) {
        const int64_t x = ccol[i];
        if (x >= lo && x < hi) atomicOr(s_row + ((x - lo) >> 5), 1u << (x & 31));
    }
    __syncthreads();
    uint32_t *row = bits + h * words + w0;
    for (int64_t w = threadIdx.x; w < nw; w += kHubThreads) row[w] = s_row[w];
}

// Inserts every arc (x -> y) into the table of x with compare-and-swap; the
// tables' contents are deterministic, their slot layout is not.
constexpr int kVtabItems = 8;
__global__ void __launch_bounds__(256)
k_vtab_build(int64_t n, int64_t nnz, const int64_t *__restrict__ coff, const int32_t *__restrict__ ccol,
             int32_t *vtab, u64 *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool failed = false;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c * kVtabItems < nnz; c += stride) {
        const int64_t i0 = c * kVtabItems;
        int64_t lo = 0, hi = n;  // last row r with coff[r] <= i0
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (ldg_i64(coff + mid) <= i0) lo = mid;
            else hi = mid - 1;
        }
        int64_t r = lo;
        int64_t ro = ldg_i64(coff + r), rend = ldg_i64(coff + r + 1);
        for (int t = 0; t < kVtabItems; t++) {
            const int64_t i = i0 + t;
            if (i >= nnz) break;
            while (rend <= i) {
                r++;
                ro = rend;
                rend = ldg_i64(coff + r + 1);
            }
            const int32_t y = ldg_i32(ccol + i);
            const uint64_t size = static_cast<uint64_t>(2 * (rend - ro));
            int32_t *tab = vtab + 2 * ro;
            uint64_t s = vtab_start(y, size);
            bool done = false;
            for (uint64_t probe = 0; probe < size; probe++) {
                const int32_t old = atomicCAS(tab + s, kEmptyLabel, y);
                if (old == kEmptyLabel || old == y) {
                    done = true;
                    break;
                }
                s = (s + 1 == size) ? 0 : s + 1;
            }
            failed |= !done;
        }
    }
    if (failed) raise_flag(status, F_OVERFLOW);
}

static int guide_shift(uint64_t W, int64_t gcap) {
    int s = 0;
    while (s < 63 && (((W - 1) >> s) + 1) > static_cast<uint64_t>(gcap)) s++;
    return s;
}

static int build_guide(ps_graph *g, const uint64_t *P, uint64_t total, int32_t *G, int slot,
                       int *shift_out, cudaStream_t s) {
    const int64_t m = g->m;
    const int shift = guide_shift(total, g->L.gcap);
    const int64_t B = static_cast<int64_t>(((total - 1) >> shift) + 1);
    *shift_out = shift;
    (void)slot;
    // one resident wave (the loop strides over the edges)
    int occ = 0;
    PS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_guide_fill, 256, 0));
    int64_t blocks = (m + 256 * kGuideGroups - 1) / (256 * kGuideGroups);
    if (blocks > (int64_t)g->sm_count * (occ > 0 ? occ : 1)) blocks = (int64_t)g->sm_count * (occ > 0 ? occ : 1);
    k_guide_fill<<<(unsigned)blocks, 256, 0, s>>>(m, P, shift, G, B);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

int launch_vertex_totals(ps_graph *g, cudaStream_t s) {
    if (g->n <= 0) return PS_OK;
    k_vertex_totals<<<g->sm_count * 8, 256, 0, s>>>(g->n, g->dnew, g->L.hub_cap, g->tune.hub_min_degree, g->status);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

int prefix_graph(ps_graph *g, cudaStream_t s) {
    const int64_t n = g->n, m = g->m;
    const int sms = g->sm_count;
    // the prefixes P_tau, P_lambda and their totals W, Lambda were written
    // by the load step's edge-table kernel (with F_OVERFLOW if a sum passed
    // 2^64), N_1 and the hub count by its vertex pass; all were read back at
    // its end
    const uint64_t flags = g->load_flags;
    if (flags & F_TIMEOUT) return PS_ERR_TIMEOUT;
    ps_stats &S = g->stats;
    S.W = g->load_totals[0];
    S.Lambda = g->load_totals[1];
    S.N1_lo = g->load_totals[2];
    S.N1_hi = g->load_totals[3];
    S.n = n;
    S.m = m;
    S.d_max = g->d_max;
    if (flags & F_OVERFLOW) return PS_ERR_OVERFLOW;

    // guide tables (with guides off the table has at most 2 buckets)
    int tshift = 0, lshift = 0;
    if (S.W > 0) {
        int rc = build_guide(g, g->ptau, S.W, g->gtau, 4, &tshift, s);
        if (rc) return rc;
    }
    if (S.Lambda > 0) {
        int rc = build_guide(g, g->plam, S.Lambda, g->glam, 5, &lshift, s);
        if (rc) return rc;
    }
    S.tau_shift = tshift;
    S.lambda_shift = lshift;

    // the edge hash set is filled by the load step (on a side stream)
    const uint64_t eset_mask = g->L.eset_buckets > 0 ? static_cast<uint64_t>(g->L.eset_buckets - 1) : 0;

    // per-vertex hash tables
    if (g->vtab) {
        PS_CUDA_TRY(cudaMemsetAsync(g->vtab, 0xFF, sizeof(int32_t) * g->L.vtab_slots, s));
        if (g->nnz > 0) {
            int64_t chunks = (g->nnz + kVtabItems - 1) / kVtabItems;
            int64_t blocks = (chunks + 255) / 256;
            if (blocks > (int64_t)sms * 64) blocks = (int64_t)sms * 64;
            k_vtab_build<<<(unsigned)blocks, 256, 0, s>>>(n, g->nnz, g->off, g->col, g->vtab, g->status);
            PS_LAUNCH_CHECK();
        }
    }

    // hub bitmaps
    const int64_t hubs = static_cast<int64_t>(g->load_totals[4]);
    S.hubs = hubs;
    if (hubs > 0) {
        const int64_t words = g->L.hub_words;
        const int64_t chunks = (words + kHubChunkWords - 1) / kHubChunkWords;
        const int smem = static_cast<int>((words < kHubChunkWords ? words : kHubChunkWords) * sizeof(uint32_t));
        PS_CUDA_TRY(cudaFuncSetAttribute(k_hub_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_hub_rows<<<(unsigned)(hubs * chunks), kHubThreads, smem, s>>>(n - hubs, g->L.hub_bit_base, g->off, g->col,
                                                                        g->hub, words, chunks);
        PS_LAUNCH_CHECK();
    }
    // The kernels queued after the synchronisation, and the hash set build,
    // cannot fail on valid state (the hash set's load is at most 1/2, so
    // every insertion finds a slot); later calls on `stream` are ordered
    // after them.

    GraphDev &D = g->dev;
    D.eset = g->eset;
    D.eset_mask = eset_mask;
    D.vtab = g->vtab;
    D.adj_mode = g->vtab ? kAdjVtab : (g->eset ? kAdjHash : kAdjSearch);
    D.hub_bit_base = static_cast<int32_t>(g->L.hub_bit_base);
    D.off = g->off;
    D.col = g->col;
    D.rec = g->rec;
    D.ptau = g->ptau;
    D.plam = g->plam;
    D.gtau = g->gtau;
    D.glam = g->glam;
    D.hub = g->hub;
    D.W = S.W;
    D.Lambda = S.Lambda;
    D.n = n;
    D.m = m;
    D.hub_start = static_cast<int32_t>(n - hubs);
    D.hub_words = static_cast<int32_t>(g->L.hub_words);
    D.tau_shift = tshift;
    D.lam_shift = lshift;
    // the hash set build of the load step ran beside everything above; later
    // calls on `s` come after it too
    const int rc = wait_eset(g, s);
    if (rc) return rc;
    g->prefixed = true;
    return (S.W == 0 || S.Lambda == 0) ? PS_NO_PATHS : PS_OK;
}

}  // namespace ps
