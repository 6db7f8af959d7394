// ps_exact.cu -- ps_count_exact: exact 4-vertex counts by enumeration, the
// ground truth that the sampled estimates are checked against where brute
// force is out of reach.  The paper gets its exact counts from separate
// enumeration code (Section 6); here they are the non-induced counts N_1..N_6
// of Eq. (1), turned into the induced counts C_1..C_6 by inverting Eq. (1):
//
//   N_1 = sum_v C(d_v, 3)            3-stars (already a total of the prefix step)
//   N_2 = W - 3 T                    W counts every 3-path once, every triangle 3 times (Section 3)
//   N_3 = sum_triangles (d_a + d_b + d_c - 6)        a triangle plus an edge at one corner
//   N_4 = 4-cycles
//   N_5 = sum_e C(t_e, 2)            two triangles sharing the chord e
//   N_6 = 4-cliques
//
// On the canonical graph (labels in degree order, rows ascending): a triangle
// a < b < c is found once, from its lowest edge (a, b), as c in the upper part
// of N(a) with c > b adjacent to b; its 4-clique extensions are the adjacent
// pairs among those c.  A 4-cycle is counted once, at its highest vertex a:
// for every opposite vertex c < a, the wedges a - b - c with b < a give
// cnt[c] common neighbours below a, and C(cnt[c], 2) cycles.
#include "ps_internal.h"

namespace ps {

namespace {

// Scratch words of the counters.
enum : int {
    XA_T = 0,        // triangles (64-bit)
    XA_N3 = 2,       // 128-bit pairs from here on
    XA_N4 = 4,
    XA_N5 = 6,
    XA_N6 = 8,
    XA_NEXT = 10,    // next vertex handed out to the 4-cycle blocks
    XA_WORDS = 16,
};

constexpr int kCliqueCap = 1024;  // common upper neighbours kept per warp in shared memory

template <int ADJ>
__device__ __forceinline__ bool has_edge(const GraphDev &g, int32_t x, int32_t y) {
    if (ADJ == kAdjHash) return eset_contains(g.eset, g.eset_mask, x, y);
    if (ADJ == kAdjVtab) {
        if (x == y) return false;
        const int32_t h = max(x, y);
        const int64_t o = ldg_i64(g.off + h);
        VtabQuery q;
        q.start(g.vtab, o, ldg_i64(g.off + h + 1) - o, min(x, y));
        return q.resolve(q.first());
    }
    return adjacent(g, x, y);
}

// First position p in col[lo, hi) with col[p] >= key.
__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *col, int64_t lo, int64_t hi, int32_t key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (ldg_i32(col + mid) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// One warp per edge (a, b), a < b.  Triangles {a, b, c}, c > b, each once;
// t_e of all three edges; the N_3 terms; then the 4-cliques {a, b, c, d}
// with c < d both such common neighbours and (c, d) an edge.
template <int ADJ>
__global__ void __launch_bounds__(256)
k_triangles_cliques(GraphDev g, const int32_t *__restrict__ lowcnt, const int64_t *__restrict__ ubase,
                    uint32_t *tcount, u64 *acc) {
    __shared__ int32_t s_common[8][kCliqueCap];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t *common = s_common[warp];
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    uint64_t tri = 0, n3lo = 0, n3hi = 0, k4 = 0;
    for (int64_t j = (int64_t)blockIdx.x * (blockDim.x / 32) + warp; j < g.m; j += nw) {
        const EdgeRec e = ldg_rec(g.rec + j);
        const int32_t a = e.u, b = e.v;
        const int64_t a_up = e.ou + ldg_i32(lowcnt + a), a_end = e.ou + e.du;
        const int32_t lb = ldg_i32(lowcnt + b);
        const int64_t b_up = e.ov + lb, b_end = e.ov + e.dv;
        const int64_t ua = ldg_i64(ubase + a), ub = ldg_i64(ubase + b);
        int found = 0;
        for (int64_t base = a_up; base < a_end; base += 32) {
            const int64_t i = base + lane;
            int32_t c = -1;
            bool in = false;
            if (i < a_end) {
                c = ldg_i32(g.col + i);
                in = c > b && has_edge<ADJ>(g, b, c);
            }
            const uint32_t mask = __ballot_sync(0xffffffffu, in);
            if (in) {
                const int pos = found + __popc(mask & lanemask_lt());
                if (pos < kCliqueCap) common[pos] = c;
                // edges (a, c) and (b, c): c sits in the upper parts of N(a) and N(b)
                const int64_t pc = lower_bound_i32(g.col, b_up, b_end, c);
                atomicAdd(tcount + ua + (i - a_up), 1u);
                atomicAdd(tcount + ub + (pc - b_up), 1u);
                const int64_t oc = ldg_i64(g.off + c);
                const uint64_t dc = static_cast<uint64_t>(ldg_i64(g.off + c + 1) - oc);
                add128(n3lo, n3hi, static_cast<uint64_t>(e.du) + static_cast<uint64_t>(e.dv) + dc - 6);
            }
            found += __popc(mask);
        }
        if (lane == 0 && found) atomicAdd(tcount + j, static_cast<uint32_t>(found));
        if (lane == 0) tri += static_cast<uint64_t>(found);
        __syncwarp();
        if (found <= kCliqueCap) {
            for (int p = 0; p + 1 < found; p++) {
                const int32_t c = common[p];
                for (int q = p + 1 + lane; q < found; q += 32) k4 += has_edge<ADJ>(g, c, common[q]) ? 1 : 0;
            }
        } else {
            // too many to keep: walk the upper part of N(a) again for each c
            for (int64_t i = a_up; i < a_end; i++) {
                const int32_t c = ldg_i32(g.col + i);
                if (c <= b || !has_edge<ADJ>(g, b, c)) continue;
                for (int64_t q = i + 1 + lane; q < a_end; q += 32) {
                    const int32_t d = ldg_i32(g.col + q);
                    k4 += (has_edge<ADJ>(g, b, d) && has_edge<ADJ>(g, c, d)) ? 1 : 0;
                }
            }
        }
        __syncwarp();
    }
    warp_add128(n3lo, n3hi);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tri += __shfl_down_sync(0xffffffffu, tri, o);
        k4 += __shfl_down_sync(0xffffffffu, k4, o);
    }
    if (lane == 0) {
        if (tri) atomicAdd(reinterpret_cast<unsigned long long *>(acc + XA_T), tri);
        if (n3lo | n3hi) atomic_add128(acc + XA_N3, n3lo, n3hi);
        if (k4) atomic_add128(acc + XA_N6, k4, 0);
    }
}

// N_5 = sum_e C(t_e, 2).
__global__ void __launch_bounds__(256) k_triangle_pairs(int64_t m, const uint32_t *__restrict__ tcount, u64 *acc) {
    uint64_t lo = 0, hi = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const uint64_t t = tcount[j];
        if (t > 1) add128(lo, hi, t * (t - 1) / 2);
    }
    warp_add128(lo, hi);
    if ((threadIdx.x & 31) == 0 && (lo | hi)) atomic_add128(acc + XA_N5, lo, hi);
}

// 4-cycles at their highest vertex a, one block per a (highest labels, the
// busiest, first).  cnt is this block's slice of n counters, all zero between
// vertices: the first pass counts the wedges a - b - c (b, c < a), the second
// takes each cnt[c] once (exchange with zero) and adds C(cnt[c], 2).
__global__ void __launch_bounds__(256)
k_cycles4(GraphDev g, const int32_t *__restrict__ lowcnt, int32_t *cnt_all, u64 *acc) {
    __shared__ int64_t s_next;
    int32_t *cnt = cnt_all + static_cast<int64_t>(blockIdx.x) * g.n;
    uint64_t lo = 0, hi = 0;
    while (true) {
        if (threadIdx.x == 0)
            s_next = static_cast<int64_t>(atomicAdd(reinterpret_cast<unsigned long long *>(acc + XA_NEXT), 1ull));
        __syncthreads();
        const int64_t k = s_next;
        __syncthreads();
        if (k >= g.n) break;
        const int32_t a = static_cast<int32_t>(g.n - 1 - k);
        const int64_t oa = ldg_i64(g.off + a);
        const int32_t la = ldg_i32(lowcnt + a);
        for (int pass = 0; pass < 2; pass++) {
            for (int idx = threadIdx.x; idx < la; idx += blockDim.x) {
                const int32_t b = ldg_i32(g.col + oa + idx);
                const int64_t ob = ldg_i64(g.off + b);
                const int64_t eb = ldg_i64(g.off + b + 1);
                // N(b) below a: a sits in the upper part of N(b)
                const int64_t pa = lower_bound_i32(g.col, ob + ldg_i32(lowcnt + b), eb, a);
                for (int64_t t = ob; t < pa; t++) {
                    const int32_t c = ldg_i32(g.col + t);
                    if (pass == 0) {
                        atomicAdd(cnt + c, 1);
                    } else {
                        const uint64_t v = static_cast<uint32_t>(atomicExch(cnt + c, 0));
                        if (v > 1) add128(lo, hi, v * (v - 1) / 2);
                    }
                }
            }
            __syncthreads();
        }
    }
    warp_add128(lo, hi);
    if ((threadIdx.x & 31) == 0 && (lo | hi)) atomic_add128(acc + XA_N4, lo, hi);
}

template <int ADJ>
int launch_triangles(const ps_graph *g, uint32_t *tcount, u64 *acc, cudaStream_t s) {
    k_triangles_cliques<ADJ><<<g->sm_count * 8, 256, 0, s>>>(g->dev, g->lowcnt, g->ubase, tcount, acc);
    PS_LAUNCH_CHECK();
    return PS_OK;
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct ExactLayout {
    size_t tcount, acc, cnt, fixed;
};

ExactLayout exact_layout(int64_t m) {
    ExactLayout L;
    L.tcount = 0;
    L.acc = align256(static_cast<size_t>(m > 0 ? m : 1) * sizeof(uint32_t));
    L.cnt = L.acc + align256(XA_WORDS * sizeof(uint64_t));
    L.fixed = L.cnt;
    return L;
}

using u128 = unsigned __int128;
using i128 = __int128;

}  // namespace

}  // namespace ps

using namespace ps;

extern "C" size_t ps_exact_scratch_bytes(const ps_graph *g, int max_blocks) {
    if (!g || !g->prefixed) return 0;
    const ExactLayout L = exact_layout(g->m);
    const int blocks = max_blocks > 0 ? max_blocks : 2 * g->sm_count;
    return L.fixed + static_cast<size_t>(blocks) * static_cast<size_t>(g->n > 0 ? g->n : 1) * sizeof(int32_t);
}

extern "C" int ps_count_exact(const ps_graph *g, void *d_scratch, size_t scratch_bytes, ps_stream_t stream,
                              uint64_t N[6], int64_t C[6]) {
    if (!g || !N || !C) return PS_ERR_ARG;
    if (!g->prefixed) return PS_ERR_STATE;
    const ExactLayout L = exact_layout(g->m);
    const size_t per_block = static_cast<size_t>(g->n > 0 ? g->n : 1) * sizeof(int32_t);
    if (!d_scratch || (reinterpret_cast<uintptr_t>(d_scratch) & 255u) != 0 ||
        scratch_bytes < L.fixed + per_block)
        return PS_ERR_WORKSPACE;
    int blocks = static_cast<int>((scratch_bytes - L.fixed) / per_block);
    if (blocks > 2 * g->sm_count) blocks = 2 * g->sm_count;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return PS_ERR_CUDA;
    if (cur != g->device && cudaSetDevice(g->device) != cudaSuccess) return PS_ERR_CUDA;
    struct Restore {
        int dev, prev;
        ~Restore() {
            if (dev != prev) cudaSetDevice(prev);
        }
    } restore{g->device, cur};

    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *base = static_cast<char *>(d_scratch);
    uint32_t *tcount = reinterpret_cast<uint32_t *>(base + L.tcount);
    u64 *acc = reinterpret_cast<u64 *>(base + L.acc);
    int32_t *cnt = reinterpret_cast<int32_t *>(base + L.cnt);
    PS_CUDA_TRY(cudaMemsetAsync(tcount, 0, static_cast<size_t>(g->m) * sizeof(uint32_t), s));
    PS_CUDA_TRY(cudaMemsetAsync(acc, 0, XA_WORDS * sizeof(uint64_t), s));
    PS_CUDA_TRY(cudaMemsetAsync(cnt, 0, static_cast<size_t>(blocks) * per_block, s));
    if (g->m > 0) {
        int rc = PS_OK;
        switch (g->dev.adj_mode) {
            case kAdjHash: rc = launch_triangles<kAdjHash>(g, tcount, acc, s); break;
            case kAdjVtab: rc = launch_triangles<kAdjVtab>(g, tcount, acc, s); break;
            default: rc = launch_triangles<kAdjSearch>(g, tcount, acc, s); break;
        }
        if (rc) return rc;
        k_triangle_pairs<<<g->sm_count * 8, 256, 0, s>>>(g->m, tcount, acc);
        PS_LAUNCH_CHECK();
        k_cycles4<<<blocks, 256, 0, s>>>(g->dev, g->lowcnt, cnt, acc);
        PS_LAUNCH_CHECK();
    }
    uint64_t h[XA_WORDS];
    PS_CUDA_TRY(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
    PS_CUDA_TRY(cudaStreamSynchronize(s));
    auto pair = [&](int w) { return (static_cast<u128>(h[w + 1]) << 64) | h[w]; };
    const ps_stats &S = g->stats;
    const u128 T = h[XA_T];
    u128 n[7];
    n[1] = (static_cast<u128>(S.N1_hi) << 64) | S.N1_lo;
    if (static_cast<u128>(S.W) < 3 * T) return PS_ERR_OVERFLOW;  // cannot happen on a valid graph
    n[2] = static_cast<u128>(S.W) - 3 * T;
    n[3] = pair(XA_N3);
    n[4] = pair(XA_N4);
    n[5] = pair(XA_N5);
    n[6] = pair(XA_N6);
    for (int i = 1; i <= 6; i++) {
        if (n[i] >> 64) return PS_ERR_OVERFLOW;
        N[i - 1] = static_cast<uint64_t>(n[i]);
    }
    // Eq. (1) is upper triangular with unit diagonal: back-substitute
    const i128 c6 = static_cast<i128>(n[6]);
    const i128 c5 = static_cast<i128>(n[5]) - 6 * c6;
    const i128 c4 = static_cast<i128>(n[4]) - c5 - 3 * c6;
    const i128 c3 = static_cast<i128>(n[3]) - 4 * c5 - 12 * c6;
    const i128 c2 = static_cast<i128>(n[2]) - 2 * c3 - 4 * c4 - 6 * c5 - 12 * c6;
    const i128 c1 = static_cast<i128>(n[1]) - c3 - 2 * c5 - 4 * c6;
    const i128 c[6] = {c1, c2, c3, c4, c5, c6};
    for (int i = 0; i < 6; i++) {
        if (c[i] > static_cast<i128>(INT64_MAX) || c[i] < static_cast<i128>(INT64_MIN)) return PS_ERR_OVERFLOW;
        C[i] = static_cast<int64_t>(c[i]);
    }
    return PS_OK;
}
