// ps_static.cu -- ps_prefix_pairs_static: the exact uint64 prefix scan of
// two weight arrays (the same single-pass scan that builds the tau / lambda
// prefixes) for callers that cannot allocate device memory.  Its scratch --
// the scan's tile flags, tile sums and tile counter -- lives in one
// fixed-size array in this file instead of a caller's workspace.
#include <cuda.h>

#include <mutex>

#include "ps_internal.h"

namespace ps {
namespace {

constexpr int64_t kStaticMaxItems = PS_PREFIX_STATIC_MAX_ITEMS;
constexpr int64_t kStaticTiles = (kStaticMaxItems + kScanTile - 1) / kScanTile;
constexpr size_t kStatusBytes = ST_WORDS * sizeof(uint64_t);
constexpr size_t kFlagBytes = ((kStaticTiles + 1) * sizeof(uint32_t) + 255) / 256 * 256;
constexpr size_t kSumBytes = (kStaticTiles + 1) * sizeof(U64x2);
constexpr size_t kOffFlags = kStatusBytes;
constexpr size_t kOffAgg = kOffFlags + kFlagBytes;
constexpr size_t kOffInc = kOffAgg + kSumBytes;
constexpr size_t kScratchBytes = kOffInc + kSumBytes;  // about 2.3 MB

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_prefix_scratch[kScratchBytes];

std::mutex g_mutex;
constexpr int kMaxDevices = 128;

// The array's device address, looked up once per device and context: a
// process that resets a device (or releases its primary context) gets a new
// context, in which the library's device code is loaded again and the array
// may sit elsewhere, so the cached address is only reused under the context
// it was read in.  Context ids (unlike context handles) are never reused.
struct ScratchAddr {
    unsigned long long ctx_id;
    void *ptr;
};
ScratchAddr g_scratch_addr[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Id of the context current on this thread; 0 when there is none or the
// driver cannot say (the address is then looked up again).
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the array on the current device (the host-side name is
// only a stand-in for it).
int scratch_address(void **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    const unsigned long long id = current_context_id();
    ScratchAddr &c = g_scratch_addr[dev];
    if (id == 0 || c.ctx_id != id || !c.ptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_prefix_scratch) != cudaSuccess || !p) return PS_ERR_CUDA;
        // the lookup itself makes the device's context current when none was
        c.ctx_id = current_context_id();
        c.ptr = p;
    }
    *out = c.ptr;
    return PS_OK;
}

struct LoadPairs {
    const uint64_t *a, *b;
    __device__ U64x2 operator()(int64_t i) const { return U64x2{a[i], b[i]}; }
};

// Inclusive prefixes; a sum that wraps past 2^64 is flagged at the first
// item where it happens (its inclusive value drops below its exclusive one).
struct StorePairs {
    uint64_t *pa, *pb;
    u64 *status;
    __device__ void operator()(int64_t i, U64x2 exc, U64x2 inc) const {
        pa[i] = inc.a;
        pb[i] = inc.b;
        if (inc.a < exc.a || inc.b < exc.b) raise_flag(status, F_OVERFLOW);
    }
};

}  // namespace
}  // namespace ps

using namespace ps;

extern "C" int ps_prefix_pairs_static(const uint64_t *d_a, const uint64_t *d_b, uint64_t *d_pa,
                                      uint64_t *d_pb, int64_t count, ps_stream_t stream) {
    if (count < 0 || (count > 0 && (!d_a || !d_b || !d_pa || !d_pb))) return PS_ERR_ARG;
    if (count > kStaticMaxItems) return PS_ERR_TOO_LARGE;
    if (count == 0) return PS_OK;
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != PS_OK) return rc;
    char *p = static_cast<char *>(base);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t tiles = (count + kScanTile - 1) / kScanTile;
    // the array keeps the previous call's contents: clear the status words,
    // the tile counter and the flags this call will use
    PS_CUDA_TRY(cudaMemsetAsync(p, 0, kStatusBytes, s));
    PS_CUDA_TRY(cudaMemsetAsync(p + kOffFlags, 0, sizeof(uint32_t) * (tiles + 1), s));
    ScanState<U64x2> st;
    st.status = reinterpret_cast<u64 *>(p);
    st.counter = reinterpret_cast<uint32_t *>(st.status + ST_COUNTER);
    st.flag = reinterpret_cast<uint32_t *>(p + kOffFlags);
    st.agg = reinterpret_cast<U64x2 *>(p + kOffAgg);
    st.inc = reinterpret_cast<U64x2 *>(p + kOffInc);
    k_scan<U64x2, kScanBlock, kScanItems><<<(unsigned)tiles, kScanBlock, 0, s>>>(
        count, st, U64x2{0, 0}, OpSum(), LoadPairs{d_a, d_b}, StorePairs{d_pa, d_pb, st.status});
    PS_LAUNCH_CHECK();
    uint64_t flags = 0;
    PS_CUDA_TRY(cudaMemcpyAsync(&flags, p, sizeof(flags), cudaMemcpyDeviceToHost, s));
    PS_CUDA_TRY(cudaStreamSynchronize(s));
    return flags_to_status(flags);
}
