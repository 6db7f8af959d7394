// ps_sample.cuh -- one draw of Alg. 1 (sample) and of Alg. 3
// (sample-centered), classified as in Alg. 2 / Alg. 4.
//
// Draw rules (identical to the CPU replay): sample `id` reads Philox block 0
// of counter (id, 0, sampler); the edge draw r uniform in [0, W) takes words
// 0-1, the neighbour draws words 2 and 3 (Lemire, rejected attempts walk
// blocks 1, 2, ...).  The edge is the first j with P[j] > r.
#pragma once

#include "ps_device.cuh"

namespace ps {

// Alg. 1 up to the induced subgraph: the edge e drawn with probability
// tau_e / W and the two neighbours u' (of u, not v) and v' (of v, not u).
__device__ __forceinline__ void path3_draw(const GraphDev &g, uint64_t seed, uint64_t id, EdgeRec &e, int32_t &up,
                                           int32_t &vp) {
    const uint4 w = sample_block(seed, id, 0, 0);
    uint64_t r;
    if (!lemire64((static_cast<uint64_t>(w.y) << 32) | w.x, g.W, r)) r = draw_r_retry(seed, id, 0, g.W);
    const int64_t j = find_edge(g.ptau, g.gtau, g.tau_shift, r);
    e = ldg_rec(g.rec + j);
    // u' uniform over N(u) \ {v}: a in [0, d_u - 1), the slot of v maps to the last entry
    const uint32_t su = static_cast<uint32_t>(e.du - 1), sv = static_cast<uint32_t>(e.dv - 1);
    uint32_t a, b;
    if (!lemire32(w.z, su, a)) a = draw_small_retry(seed, id, 0, 2, su);
    if (!lemire32(w.w, sv, b)) b = draw_small_retry(seed, id, 0, 3, sv);
    const int32_t pa = (a == static_cast<uint32_t>(e.iu)) ? e.du - 1 : static_cast<int32_t>(a);
    const int32_t pb = (b == static_cast<uint32_t>(e.jv)) ? e.dv - 1 : static_cast<int32_t>(b);
    up = ldg_i32(g.col + e.ou + pa);
    vp = ldg_i32(g.col + e.ov + pb);
}

// Class of a 3-path u'-u-v-v' (u' != v') from its three other pairs
// (u', v), (u, v'), (u', v'): 1 = 3-path, 2 = tailed triangle, 3 = 4-cycle,
// 4 = chordal 4-cycle, 5 = 4-clique.
__device__ __forceinline__ int class3(bool e1, bool e2, bool e3) {
    const int s = (int)e1 + (int)e2 + (int)e3;
    return s == 0 ? 1 : (s == 1 ? (e3 ? 3 : 2) : (s == 2 ? 4 : 5));
}

// Class of one Alg. 1 output: 0 = triangle (u' == v'), 1 = 3-path,
// 2 = tailed triangle, 3 = 4-cycle, 4 = chordal 4-cycle, 5 = 4-clique.
// HUB_ALL: every adjacency test of a sample may read a hub row (see
// pair_test3); false for kernels short of registers.
template <int ADJ, bool HUB_ALL = true>
__device__ __forceinline__ int sample_3path(const GraphDev &g, uint64_t seed, uint64_t id) {
    EdgeRec e;
    int32_t up, vp;
    path3_draw(g, seed, id, e, up, vp);
    if (up == vp) return 0;
    // the path u'-u-v-v' is present; the pairs (u',v), (u,v'), (u',v') decide
    bool e1, e2, e3;
    if (ADJ == kAdjHash) {
        pair_test3<HUB_ALL>(g, up, e.v, e.u, vp, up, vp, e1, e2, e3);
    } else if (ADJ == kAdjVtab) {
        // (u', v) in the table of v, (u, v') in the table of u -- both rows
        // are in the edge record -- and (u', v') in the larger label's table
        const int32_t x3 = max(up, vp);
        const int64_t o3 = ldg_i64(g.off + x3);
        const int64_t d3 = ldg_i64(g.off + x3 + 1) - o3;
        VtabQuery q1, q2, q3;
        q1.start(g.vtab, e.ov, e.dv, up);
        q2.start(g.vtab, e.ou, e.du, vp);
        q3.start(g.vtab, o3, d3, min(up, vp));
        const int32_t f1 = q1.first(), f2 = q2.first(), f3 = q3.first();
        e1 = q1.resolve(f1);
        e2 = q2.resolve(f2);
        e3 = q3.resolve(f3);
    } else {
        e1 = (up < e.v) ? adjacent(g, up, e.v) : adjacent_known(g, e.v, e.ov, e.dv, up);
        e2 = (e.u < vp) ? adjacent_known(g, e.u, e.ou, e.du, vp) : adjacent(g, vp, e.u);
        e3 = adjacent(g, up, vp);
    }
    return class3(e1, e2, e3);
}

// Alg. 3 up to the induced subgraph: the edge e drawn with probability
// lambda_e / Lambda, u' among the L_{u,v} entries of N(u) after v and v'
// among the L_{v,u} entries of N(v) after u.
__device__ __forceinline__ void centred_draw(const GraphDev &g, uint64_t seed, uint64_t id, EdgeRec &e, int32_t &up,
                                             int32_t &vp) {
    const uint4 w = sample_block(seed, id, 0, 1);
    uint64_t r;
    if (!lemire64((static_cast<uint64_t>(w.y) << 32) | w.x, g.Lambda, r))
        r = draw_r_retry(seed, id, 1, g.Lambda);
    const int64_t j = find_edge(g.plam, g.glam, g.lam_shift, r);
    e = ldg_rec(g.rec + j);
    const uint32_t lu = static_cast<uint32_t>(e.du - 1 - e.iu);
    const uint32_t lv = static_cast<uint32_t>(e.dv - 1 - e.jv);
    uint32_t a, b;
    if (!lemire32(w.z, lu, a)) a = draw_small_retry(seed, id, 1, 2, lu);
    if (!lemire32(w.w, lv, b)) b = draw_small_retry(seed, id, 1, 3, lv);
    up = ldg_i32(g.col + e.ou + e.iu + 1 + static_cast<int32_t>(a));
    vp = ldg_i32(g.col + e.ov + e.jv + 1 + static_cast<int32_t>(b));
}

// Class of one Alg. 3 output: 0 = not centred, 1 = 4-cycle, 2 = chordal
// 4-cycle, 3 = 4-clique.  u' is drawn among the L_{u,v} entries of N(u)
// after v, v' among the L_{v,u} entries of N(v) after u; the path is centred
// (Definition 4.1) iff (u', v') is an edge.
template <int ADJ, bool HUB_ALL = true>
__device__ __forceinline__ int sample_centred(const GraphDev &g, uint64_t seed, uint64_t id) {
    EdgeRec e;
    int32_t up, vp;
    centred_draw(g, seed, id, e, up, vp);
    if (ADJ == kAdjVtab) {
        if (up == vp) return 0;
        // the chords (u', v) and (u, v') in the tables of v and u (rows known
        // from the record, looked up alongside), the closing edge (u', v') in
        // the larger label's table
        const int32_t x = max(up, vp);
        const int64_t ox = ldg_i64(g.off + x);
        const int64_t dx = ldg_i64(g.off + x + 1) - ox;
        VtabQuery q0, q1, q2;
        q1.start(g.vtab, e.ov, e.dv, up);
        q2.start(g.vtab, e.ou, e.du, vp);
        q0.start(g.vtab, ox, dx, min(up, vp));
        const int32_t f1 = q1.first(), f2 = q2.first(), f0 = q0.first();
        if (!q0.resolve(f0)) return 0;  // not centred
        return 1 + (int)q1.resolve(f1) + (int)q2.resolve(f2);
    }
    if (ADJ == kAdjHash) {
        // the closing edge first; the two chords only for centred paths
        if (!pair_test(g, up, vp)) return 0;  // also u' == v'
        bool c1, c2;
        pair_test2<HUB_ALL>(g, e.v, up, e.u, vp, c1, c2);
        return 1 + (int)c1 + (int)c2;
    }
    if (!adjacent(g, up, vp)) return 0;  // also covers u' == v'
    // u' > v and v' > u in label order, so the chord tests search N(v) and N(u)
    const bool c1 = adjacent_known(g, e.v, e.ov, e.dv, up);
    const bool c2 = adjacent_known(g, e.u, e.ou, e.du, vp);
    return 1 + (int)c1 + (int)c2;
}

// Registers for 768 resident threads per SM (three blocks of 256, 85
// registers): the hub-row tests otherwise take 98 and drop to two blocks
// (3-path sampling on R-MAT 20: 1.61 ms capped, 1.74 ms not).  Blocks of 512
// and 1024 keep the compiler's choice.
template <int BLOCK>
constexpr int sample_min_blocks() { return BLOCK <= 256 ? 768 / BLOCK : 1; }

// Per-thread class counters kept in registers.
struct Counts6 {
    uint32_t c[6];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < 6; i++) c[i] = 0;
    }
    __device__ __forceinline__ void add(int cls) {
#pragma unroll
        for (int i = 0; i < 6; i++) c[i] += (cls == i);
    }
};

// Block-wide sum of the counters, added to hist[0..nbins) with one atomic per
// bin per block.
template <int BLOCK>
__device__ __forceinline__ void flush_counts(Counts6 &cnt, int nbins, uint64_t *hist) {
    __shared__ unsigned long long s_bins[6];
    if (threadIdx.x < 6) s_bins[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 6; i++) {
        unsigned long long x = cnt.c[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_bins[i], x);
    }
    __syncthreads();
    if (threadIdx.x < nbins && s_bins[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long *>(hist + threadIdx.x), s_bins[threadIdx.x]);
    __syncthreads();
}

}  // namespace ps
