// Top-k selection (Sec. 1: the k nodes with the highest similarity to the source).
//
// Each candidate node i gets a 96-bit key (ordered(score) << 32 | ~i): a larger
// key is a higher score, and among equal scores a smaller id.  Keys are unique,
// so the top-k set is unique.  A most-significant-digit radix select (8-bit
// digits, warp-aggregated shared-memory histograms) narrows a key prefix until
// the bucket at the current depth holds exactly the number of keys still
// needed; every key at or above that prefix is selected, and one block sorts
// the <= 4096 winners (bitonic, shared memory).
#include "common.cuh"
#include "internal.h"
#include "exactsim.h"
#include <cuda.h>

#include <mutex>
#include <string>

namespace esim {

namespace {

struct TopkState {
    unsigned long long pre_hi;
    unsigned int pre_lo;
    unsigned int k_rem;
    int depth;      // number of 8-bit digits fixed in the prefix
    int done;
    unsigned int count;
    unsigned int pad;
    unsigned int hist[256];
};

struct Cand {
    unsigned long long hi;
    unsigned int lo;
    unsigned int pad;
};

__device__ __forceinline__ unsigned long long ordered_bits(double s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(s);
    return (b >> 63) ? ~b : (b ^ 0x8000000000000000ull);
}

__device__ __forceinline__ double from_ordered(unsigned long long o) {
    const unsigned long long b = (o >> 63) ? (o ^ 0x8000000000000000ull) : ~o;
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ unsigned digit_of(unsigned long long hi, unsigned lo, int d) {
    return d < 8 ? (unsigned)((hi >> (56 - 8 * d)) & 0xFFu) : (unsigned)((lo >> (24 - 8 * (d - 8))) & 0xFFu);
}

// Compare the top `depth` digits of (hi, lo) with the prefix: -1, 0, +1.
__device__ __forceinline__ int cmp_prefix(unsigned long long hi, unsigned lo, const TopkState& s, int depth) {
    if (depth == 0) return 0;
    if (depth <= 8) {
        const int sh = 64 - 8 * depth;
        const unsigned long long a = hi >> sh, b = s.pre_hi >> sh;
        return a < b ? -1 : (a > b ? 1 : 0);
    }
    if (hi != s.pre_hi) return hi < s.pre_hi ? -1 : 1;
    const int sh = 32 - 8 * (depth - 8);
    const unsigned a = sh >= 32 ? 0u : (lo >> sh), b = sh >= 32 ? 0u : (s.pre_lo >> sh);
    return a < b ? -1 : (a > b ? 1 : 0);
}

// Every kernel below handles one column per blockIdx.y (select/sort: blockIdx.x);
// a single selection is the one-column case.
__global__ void topk_init_kernel(TopkState* st, unsigned k) {
    st += blockIdx.x;
    const int t = threadIdx.x;
    if (t == 0) {
        st->pre_hi = 0;
        st->pre_lo = 0;
        st->k_rem = k;
        st->depth = 0;
        st->done = 0;
        st->count = 0;
    }
    for (int b = t; b < 256; b += blockDim.x) st->hist[b] = 0;
}

__global__ void __launch_bounds__(kBlock) topk_hist_kernel(int64_t n, const double* __restrict__ scores,
                                                           int64_t exclude, TopkState* __restrict__ st, int d,
                                                           int64_t col_stride, const int64_t* __restrict__ excl) {
    __shared__ unsigned int h[256];
    scores += (int64_t)blockIdx.y * col_stride;
    st += blockIdx.y;
    if (excl) exclude = excl[blockIdx.y];
    if (st->done) return;
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const TopkState s = *st;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform loop so that every lane takes part in the match below
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t i = base + lane;
        unsigned dig = 256u;  // sentinel: not counted
        if (i < n && i != exclude) {
            const unsigned long long hi = ordered_bits(scores[i]);
            const unsigned lo = ~(unsigned)i;
            if (cmp_prefix(hi, lo, s, d) == 0) dig = digit_of(hi, lo, d);
        }
        // warp-aggregated increment: one shared atomic per distinct digit in the warp
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        if (dig < 256u && lane == __ffs(peers) - 1) atomicAdd(&h[dig], (unsigned)__popc(peers));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&st->hist[b], h[b]);
}

__global__ void topk_select_kernel(TopkState* st, int d) {
    st += blockIdx.x;
    if (threadIdx.x != 0 || st->done) return;
    unsigned total = 0;
    for (int b = 0; b < 256; ++b) total += st->hist[b];
    if (d == 0 && total <= st->k_rem) {  // fewer candidates than k: take all
        st->done = 1;
        st->depth = 0;
    } else {
        unsigned cum = 0;
        int B = 0;
        for (int b = 255; b >= 0; --b) {
            const unsigned c = st->hist[b];
            if (cum + c >= st->k_rem) {
                B = b;
                break;
            }
            cum += c;
        }
        if (d < 8) st->pre_hi |= (unsigned long long)B << (56 - 8 * d);
        else st->pre_lo |= (unsigned)B << (24 - 8 * (d - 8));
        st->k_rem -= cum;
        st->depth = d + 1;
        if (st->hist[B] == st->k_rem) st->done = 1;
    }
    for (int b = 0; b < 256; ++b) st->hist[b] = 0;
}

__global__ void __launch_bounds__(kBlock) topk_gather_kernel(int64_t n, const double* __restrict__ scores,
                                                             int64_t exclude, TopkState* __restrict__ st,
                                                             Cand* __restrict__ cand, unsigned cap, int64_t col_stride,
                                                             const int64_t* __restrict__ excl) {
    scores += (int64_t)blockIdx.y * col_stride;
    st += blockIdx.y;
    cand += (size_t)blockIdx.y * cap;
    if (excl) exclude = excl[blockIdx.y];
    const TopkState s = *st;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (i == exclude) continue;
        const unsigned long long hi = ordered_bits(scores[i]);
        const unsigned lo = ~(unsigned)i;
        if (cmp_prefix(hi, lo, s, s.depth) < 0) continue;
        const unsigned slot = atomicAdd(&st->count, 1u);
        if (slot < cap) cand[slot] = Cand{hi, lo, 0u};
    }
}

// One block of 1024 threads sorts the selected keys, descending.  P (a power of
// two >= k) keys live in dynamic shared memory: P * 12 bytes <= 48 KB.
__global__ void __launch_bounds__(1024) topk_sort_kernel(const TopkState* __restrict__ st,
                                                         const Cand* __restrict__ cand, int k, int P,
                                                         int32_t* __restrict__ ids_out, double* __restrict__ vals_out,
                                                         unsigned cap) {
    extern __shared__ unsigned long long sm_hi[];
    st += blockIdx.x;
    cand += (size_t)blockIdx.x * cap;
    ids_out += (size_t)blockIdx.x * k;
    vals_out += (size_t)blockIdx.x * k;
    unsigned* sm_lo = (unsigned*)(sm_hi + P);
    unsigned cnt = st->count;
    if (cnt > (unsigned)k) cnt = (unsigned)k;  // cannot happen for unique keys; guards the buffer
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const bool real = i < (int)cnt;
        sm_hi[i] = real ? cand[i].hi : 0ull;  // (0, 0) is below every real key (ids < 2^31)
        sm_lo[i] = real ? cand[i].lo : 0u;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const unsigned long long ah = sm_hi[i], bh = sm_hi[j];
                    const unsigned al = sm_lo[i], bl = sm_lo[j];
                    const bool a_less = ah < bh || (ah == bh && al < bl);
                    const bool desc = (i & size) == 0;  // overall order: descending
                    if (desc ? a_less : !a_less) {
                        sm_hi[i] = bh;
                        sm_hi[j] = ah;
                        sm_lo[i] = bl;
                        sm_lo[j] = al;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        if (i < (int)cnt) {
            ids_out[i] = (int32_t)(~sm_lo[i]);
            vals_out[i] = from_ordered(sm_hi[i]);
        } else {
            ids_out[i] = -1;
            vals_out[i] = 0.0;
        }
    }
}

}  // namespace

size_t topk_workspace_bytes(int64_t /*n*/) { return sizeof(TopkState) + sizeof(Cand) * (size_t)kTopkMax + 256; }

cudaError_t launch_topk(const Graph& g, const double* scores, int64_t exclude, int32_t k, int32_t* ids_out,
                        double* vals_out, void* ws) {
    TopkState* st = (TopkState*)ws;
    Cand* cand = (Cand*)((char*)ws + ((sizeof(TopkState) + 255) / 256) * 256);
    topk_init_kernel<<<1, 256, 0, g.stream>>>(st, (unsigned)k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t blocks = (g.n + kBlock - 1) / kBlock;
    if (blocks > (int64_t)g.sm_count * 4) blocks = (int64_t)g.sm_count * 4;
    if (blocks < 1) blocks = 1;
    for (int d = 0; d < 12; ++d) {
        topk_hist_kernel<<<(unsigned)blocks, kBlock, 0, g.stream>>>(g.n, scores, exclude, st, d, 0, nullptr);
        topk_select_kernel<<<1, 32, 0, g.stream>>>(st, d);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    topk_gather_kernel<<<(unsigned)blocks, kBlock, 0, g.stream>>>(g.n, scores, exclude, st, cand, (unsigned)kTopkMax, 0,
                                                                  nullptr);
    int P = 1;
    while (P < k) P <<= 1;
    topk_sort_kernel<<<1, 1024, (size_t)P * 12, g.stream>>>(st, cand, k, P, ids_out, vals_out, (unsigned)kTopkMax);
    return cudaGetLastError();
}

size_t topk_batch_workspace_bytes(int32_t B) {
    return ((sizeof(TopkState) * (size_t)B + 255) / 256) * 256 + sizeof(Cand) * (size_t)kTopkMax * (size_t)B;
}

// B independent selections: column q of scores starts at scores + q * n; exclude[q]
// (device, may be NULL for none) is left out of column q.
cudaError_t launch_topk_batch(const Graph& g, int32_t B, const double* scores, const int64_t* exclude, int32_t k,
                              int32_t* ids_out, double* vals_out, void* ws) {
    TopkState* st = (TopkState*)ws;
    Cand* cand = (Cand*)((char*)ws + ((sizeof(TopkState) * (size_t)B + 255) / 256) * 256);
    topk_init_kernel<<<(unsigned)B, 256, 0, g.stream>>>(st, (unsigned)k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t blocks = (g.n + kBlock - 1) / kBlock;
    int64_t cap = ((int64_t)g.sm_count * 4 + B - 1) / B;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const dim3 grid((unsigned)blocks, (unsigned)B);
    for (int d = 0; d < 12; ++d) {
        topk_hist_kernel<<<grid, kBlock, 0, g.stream>>>(g.n, scores, -1, st, d, g.n, exclude);
        topk_select_kernel<<<(unsigned)B, 32, 0, g.stream>>>(st, d);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    topk_gather_kernel<<<grid, kBlock, 0, g.stream>>>(g.n, scores, -1, st, cand, (unsigned)kTopkMax, g.n, exclude);
    int P = 1;
    while (P < k) P <<= 1;
    topk_sort_kernel<<<(unsigned)B, 1024, (size_t)P * 12, g.stream>>>(st, cand, k, P, ids_out, vals_out,
                                                                     (unsigned)kTopkMax);
    return cudaGetLastError();
}

}  // namespace esim

// ---------------------------------------------------------------------------
// Top-k selection that allocates nothing (esim_select_topk_static).
//
// Some callers cannot call cudaMalloc: code that runs inside a host framework
// which owns every byte of device memory (a fixed arena or a memory-capped
// serving process), and latency-critical threads that must not pay the device
// synchronisation cudaMalloc/cudaFree may cause.  For them the selection's
// scratch (its radix-select state and the candidate list, about 66 KB) lives in
// the file-scope array below instead of a library or caller allocation.  Every
// GPU that loads the library holds this array until the process exits.
//
// In host code the symbol `g_topk_static_scratch` is only a host-side stand-in:
// passing it to a kernel would fault or, where the GPU can reach host memory,
// silently use the wrong memory.  The device address is taken once per device
// with cudaGetSymbolAddress (the first call on a device does this, with that
// device current; make that first call before any stream capture) and passed to
// the kernels.  The address is remembered together with the unique id of the CUDA
// context it was taken in: after a device reset the device has a new context (and
// the array a new address), so the next call takes the address again.  All calls
// share the array and it keeps the last call's contents; topk_init_kernel clears
// the state every call.  Calls whose work overlaps on the GPU (different streams,
// or several host threads) race on the array.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kStaticTopkStateBytes = ((sizeof(esim::TopkState) + 255) / 256) * 256;
constexpr size_t kStaticTopkScratchBytes = kStaticTopkStateBytes + sizeof(esim::Cand) * (size_t)esim::kTopkMax;

static __device__ __align__(256) unsigned char g_topk_static_scratch[kStaticTopkScratchBytes];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {};
int g_static_sms[kStaticMaxDevices] = {};
unsigned long long g_static_ctx[kStaticMaxDevices] = {};  // context id the address belongs to

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the CUDA context current on this thread, from the driver's entry points.
// With no context current yet, the device's primary context is made current first (the
// context the runtime would use); a context the caller made current is left alone.
cudaError_t current_context_id(int dev, unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f0 = nullptr;
        void* f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0);
        if (e != cudaSuccess) return e;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return cudaErrorNotSupported;
        get_current = (CtxGetCurrentFn)f0;
        get_id = (CtxGetIdFn)f1;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    if (!ctx) {
        cudaError_t e = cudaSetDevice(dev);
        if (e != cudaSuccess) return e;
        if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
    }
    if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

// Device address of the scratch array and the SM count of the current device, taken
// again whenever the device's context differs from the one they were taken in.
cudaError_t static_scratch(int dev, void** ptr, int* sms) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    unsigned long long ctx = 0;
    cudaError_t e = current_context_id(dev, &ctx);
    if (e != cudaSuccess) return e;
    if (!g_static_ptr[dev] || g_static_ctx[dev] != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_topk_static_scratch);
        if (e != cudaSuccess) return e;
        int s = 0;
        e = cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_static_sms[dev] = s;
        g_static_ptr[dev] = p;
        g_static_ctx[dev] = ctx;
    }
    *ptr = g_static_ptr[dev];
    *sms = g_static_sms[dev];
    return cudaSuccess;
}

esim_status static_fail(esim_status status, const std::string& message) {
    esim::set_error((int)status, message);
    return status;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) esim_status esim_select_topk_static(
    const double* scores, int64_t n, int64_t exclude, int32_t k, int32_t* ids_out, double* vals_out, void* stream) {
    using namespace esim;
    if (!scores || !ids_out || !vals_out) return static_fail(ESIM_EINVAL, "NULL argument");
    if (n < 1 || n >= ((int64_t)1 << 31)) return static_fail(ESIM_EINVAL, "need 1 <= n < 2^31");
    if (k < 1) return static_fail(ESIM_EINVAL, "k must be >= 1");
    if (k > kTopkMax)
        return static_fail(ESIM_ENOTSUP, "k above 4096: the static top-k scratch holds at most 4096 candidates");
    if (exclude < -1 || exclude >= n) return static_fail(ESIM_EINVAL, "exclude out of range");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return static_fail(ESIM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kStaticMaxDevices) return static_fail(ESIM_ENOTSUP, "device ordinal above 63");
    void* ws = nullptr;
    int sms = 0;
    e = static_scratch(dev, &ws, &sms);
    if (e != cudaSuccess)
        return static_fail(ESIM_ECUDA, std::string("static scratch set-up: ") + cudaGetErrorString(e));
    cudaStream_t st = (cudaStream_t)stream;
    TopkState* state = (TopkState*)ws;
    Cand* cand = (Cand*)((char*)ws + kStaticTopkStateBytes);
    topk_init_kernel<<<1, 256, 0, st>>>(state, (unsigned)k);
    int64_t blocks = (n + kBlock - 1) / kBlock;
    if (blocks > (int64_t)sms * 4) blocks = (int64_t)sms * 4;
    if (blocks < 1) blocks = 1;
    for (int d = 0; d < 12; ++d) {
        topk_hist_kernel<<<(unsigned)blocks, kBlock, 0, st>>>(n, scores, exclude, state, d, 0, nullptr);
        topk_select_kernel<<<1, 32, 0, st>>>(state, d);
    }
    topk_gather_kernel<<<(unsigned)blocks, kBlock, 0, st>>>(n, scores, exclude, state, cand, (unsigned)kTopkMax, 0,
                                                              nullptr);
    int P = 1;
    while (P < k) P <<= 1;
    topk_sort_kernel<<<1, 1024, (size_t)P * 12, st>>>(state, cand, k, P, ids_out, vals_out, (unsigned)kTopkMax);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(ESIM_ECUDA, std::string("static top-k launch: ") + cudaGetErrorString(e));
    return ESIM_OK;
}
