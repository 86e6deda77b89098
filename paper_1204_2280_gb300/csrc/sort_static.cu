// sort_static.cu -- bonsai_sort_keys_static: the stable radix sort of 63-bit
// keys with all of its scratch in one file-scope device array, for callers
// that must not allocate device memory.
//
// Who needs this: code that cannot call cudaMalloc/cudaFree around a sort --
// a latency-critical loop (cudaMalloc and cudaFree can synchronise the whole
// device and take milliseconds), or a host application whose own caching
// allocator has already reserved the device memory (a second allocator would
// fail or fragment it).  Such a caller passes its own input and output
// buffers and this entry point takes nothing else from the device heap.
// The call reads a status word back and synchronises its stream before it
// returns, so it cannot be recorded into a CUDA graph by stream capture.
//
// The scratch (about 0.9 MiB) is a static __device__ array: every GPU on
// which the library is loaded holds it until the process exits, and every
// call shares it.  Calls whose GPU work overlaps (two host threads, or two
// streams) would race on it, so callers must serialise them.
#include <mutex>

#include "common.cuh"

namespace bonsai {

__global__ void k_onesweep(const unsigned long long *__restrict__ kin, const uint32_t *__restrict__ vin,
                           unsigned long long *__restrict__ kout, uint32_t *__restrict__ vout, int n,
                           int shift, const unsigned *__restrict__ ghist, unsigned *status,
                           unsigned *status_next, unsigned *ticket, int ntiles, DevState *st,
                           long long max_spin, const uint8_t *__restrict__ dsrc);
extern const size_t SORT_DYN_SMEM_BYTES;

constexpr int STATIC_SORT_MAX_N = 1 << 16;                       // 65536 keys
constexpr int STATIC_SORT_TILES = STATIC_SORT_MAX_N / SORT_TILE;  // 16 tiles

struct StaticSortScratch {
    DevState st;                                                 // histograms, tickets, status
    unsigned long long keys_alt[STATIC_SORT_MAX_N];
    uint32_t vals_alt[STATIC_SORT_MAX_N];
    unsigned tile_status[SORT_PASSES * STATIC_SORT_TILES * SORT_RADIX];
};

// Device-resident scratch.  Host code must never pass this name to a kernel:
// on the host it is only a stand-in; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) StaticSortScratch g_sort_scratch;

// Clears everything a sort must find at zero, then builds the 8 digit
// histograms of the keys.
__global__ void k_static_clear(StaticSortScratch *s) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = t; i < SORT_PASSES * SORT_RADIX; i += gridDim.x * blockDim.x) s->st.hist[i] = 0u;
    for (int i = t; i < STATIC_SORT_TILES * SORT_RADIX; i += gridDim.x * blockDim.x) s->tile_status[i] = 0u;
    if (t < SORT_PASSES) s->st.sort_tile[t] = 0u;
    if (t == 0) { s->st.status = 0u; s->st.hold_tile = 0u; }
}

__global__ void k_static_hist(const unsigned long long *__restrict__ keys, int n, StaticSortScratch *s) {
    __shared__ unsigned h[SORT_PASSES * SORT_RADIX];
    for (int i = threadIdx.x; i < SORT_PASSES * SORT_RADIX; i += blockDim.x) h[i] = 0u;
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned long long k = keys[i];
#pragma unroll
        for (int d = 0; d < SORT_PASSES; d++)
            atomicAdd(&h[d * SORT_RADIX + (unsigned)((k >> (SORT_BITS * d)) & (SORT_RADIX - 1))], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SORT_PASSES * SORT_RADIX; i += blockDim.x)
        if (h[i]) atomicAdd(&s->st.hist[i], h[i]);
}

void set_global_error(const char *msg);   // api.cu: text of bonsai_last_error(NULL)

namespace {
std::mutex g_setup_mu;
StaticSortScratch *g_dev_ptr[MAX_DEVICES] = {};

int set_err(int code, const char *msg) {
    cudaGetLastError();
    set_global_error(msg);
    return code;
}
}  // namespace

}  // namespace bonsai

using namespace bonsai;

extern "C" int bonsai_sort_keys_static(const uint64_t *keys, uint64_t *sorted_keys, uint32_t *perm,
                                       long long n, void *cuda_stream) {
    if (!keys || !sorted_keys || !perm || n < 1)
        return set_err(BONSAI_ERR_INVALID_ARG, "bonsai_sort_keys_static: need device keys, outputs and n >= 1");
    if (n > STATIC_SORT_MAX_N)
        return set_err(BONSAI_ERR_INVALID_ARG,
                       "bonsai_sort_keys_static: n exceeds the static scratch limit of 65536 keys");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return set_err(BONSAI_ERR_CUDA, "bonsai_sort_keys_static: no usable current device");
    StaticSortScratch *s = nullptr;
    {
        // Once per device, with that device current: the device address of
        // the static scratch, and the sort kernel's shared-memory limit (a
        // per-device attribute).
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_dev_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
            if (e != cudaSuccess || !p)
                return set_err(BONSAI_ERR_CUDA, "bonsai_sort_keys_static: cudaGetSymbolAddress failed");
            e = cudaFuncSetAttribute(k_onesweep, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)SORT_DYN_SMEM_BYTES);
            if (e != cudaSuccess)
                return set_err(BONSAI_ERR_CUDA, "bonsai_sort_keys_static: kernel attribute setup failed");
            g_dev_ptr[dev] = (StaticSortScratch *)p;
        }
        s = g_dev_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int nn = (int)n, ntiles = (nn + SORT_TILE - 1) / SORT_TILE;
    k_static_clear<<<16, 256, 0, st>>>(s);
    k_static_hist<<<16, 256, 0, st>>>((const unsigned long long *)keys, nn, s);
    // Ping-pong between the scratch and the caller's output buffers so that
    // the last pass lands in the outputs: pass p reads buffer set p (the
    // caller's keys for p = 0) and writes set p + 1, where set j >= 1 is the
    // outputs when SORT_PASSES - j is even and the scratch otherwise.
    unsigned long long *kb[2] = {(unsigned long long *)sorted_keys, s->keys_alt};
    uint32_t *vb[2] = {perm, s->vals_alt};
    const size_t plane = (size_t)STATIC_SORT_TILES * SORT_RADIX;
    for (int p = 0; p < SORT_PASSES; p++) {
        const int in_set = (SORT_PASSES - p) & 1, out_set = (SORT_PASSES - p - 1) & 1;
        const unsigned long long *kin = p == 0 ? (const unsigned long long *)keys : kb[in_set];
        const uint32_t *vin = p == 0 ? nullptr : vb[in_set];
        k_onesweep<<<ntiles, SORT_THREADS, SORT_DYN_SMEM_BYTES, st>>>(
            kin, vin, kb[out_set], vb[out_set], nn, SORT_BITS * p, s->st.hist + SORT_RADIX * p,
            s->tile_status + plane * p, p + 1 < SORT_PASSES ? s->tile_status + plane * (p + 1) : nullptr,
            s->st.sort_tile + p, ntiles, &s->st, 1ll << 24, nullptr);
    }
    if (cudaGetLastError() != cudaSuccess)
        return set_err(BONSAI_ERR_CUDA, "bonsai_sort_keys_static: kernel launch failed");
    unsigned status = 0;
    if (cudaMemcpyAsync(&status, &s->st.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return set_err(BONSAI_ERR_CUDA, "bonsai_sort_keys_static: device error");
    if (status & ST_TIMEOUT)
        return set_err(BONSAI_ERR_TIMEOUT, "bonsai_sort_keys_static: a bounded look-back wait gave up");
    return BONSAI_OK;
}
