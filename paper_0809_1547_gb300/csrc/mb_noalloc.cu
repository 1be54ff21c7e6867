// Energy sum that allocates nothing: the two-pass reduction of the field
// energy with its scratch (per-block partial sums and a non-finite flag) in
// a file-scope device array instead of memory allocated by a context.
//
// For callers that cannot allocate device memory: code that runs while a
// framework's caching allocator owns the device memory, code that must not
// pay the device-wide synchronisation cudaMalloc / cudaFree imply, and code
// under a per-process memory limit.  Every GPU that loads this library holds
// the array (kNoAllocParts doubles + one int, about 64 KB) until the process
// exits.
#include "mb_host.h"

#include <mutex>

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocCellsPerThread = 32;
constexpr int64_t kNoAllocCellsPerBlock = (int64_t)kNoAllocThreads * kNoAllocCellsPerThread;
constexpr int kNoAllocParts = 8192;                       // partial sums the array holds
constexpr int64_t kNoAllocMaxCells = kNoAllocCellsPerBlock * kNoAllocParts;   // 67,108,864

struct NoAllocScratch {
    double partial[kNoAllocParts];
    int nonfinite;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// In host code the name g_noalloc_scratch is a host-side stand-in, not a
// device address: the kernels receive the address cudaGetSymbolAddress
// returned for the current device.  That address belongs to the device's
// context; a device reset (cudaDeviceReset) replaces the context and
// reloads the module, so the cached address is kept with the context's
// process-unique id and looked up again when the id changes.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoAllocSlot {
    NoAllocScratch* ptr;
    unsigned long long ctx_id;
};
NoAllocSlot g_noalloc_slot[kMaxDevices] = {};

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);

// The current context's id (cuCtxGetId, through the runtime's driver
// entry-point query); false when there is no current context yet or the
// driver does not provide the calls.
bool current_context_id(unsigned long long* id) {
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PfnCtxGetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PfnCtxGetId>(p);
    });
    if (!get_current || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Pass 1: block b sums w |E|^2 + |H|^2 over cells [b C, (b+1) C) in FP64.
__global__ void __launch_bounds__(kNoAllocThreads)
k_energy_partial_static(const float* ex, const float* ey, const float* ez, const float* hx,
                        const float* hy, const float* hz, const float* eps_r, int64_t ncell,
                        NoAllocScratch* scratch) {
    const int64_t begin = blockIdx.x * kNoAllocCellsPerBlock;
    const int64_t end = begin + kNoAllocCellsPerBlock < ncell ? begin + kNoAllocCellsPerBlock : ncell;
    double acc = 0.0;
    bool bad = false;
    for (int64_t c = begin + threadIdx.x; c < end; c += kNoAllocThreads) {
        const float e2 = ex[c] * ex[c] + ey[c] * ey[c] + ez[c] * ez[c];
        const float h2 = hx[c] * hx[c] + hy[c] * hy[c] + hz[c] * hz[c];
        const double w = eps_r ? (double)eps_r[c] : 1.0;
        bad |= !isfinite(e2) || !isfinite(h2);
        acc += w * (double)e2 + (double)h2;
    }
    __shared__ double red[kNoAllocThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < kNoAllocThreads / 32 ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) scratch->partial[blockIdx.x] = acc;
    }
    if (bad) atomicOr(&scratch->nonfinite, 1);
}

// Pass 2: one block sums the partials in a fixed order; out = (sum, flag).
__global__ void k_energy_final_static(const NoAllocScratch* scratch, int nparts, double* out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) acc += scratch->partial[q];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            out[0] = acc;
            out[1] = scratch->nonfinite ? 1.0 : 0.0;
        }
    }
}

int noalloc_fail(int code, const std::string& msg) {
    mb::set_thread_error(msg);   // read back with mb_last_error(NULL)
    return code;
}

// Address of the array on the current device: looked up on the first call
// made with that device current, and again once the device's context has
// been replaced (the cached context id no longer matches).
int noalloc_scratch(NoAllocScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(MB_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(MB_ERR_ARG, "device index beyond 64");
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocSlot& slot = g_noalloc_slot[dev];
    if (!slot.ptr || !have_id || slot.ctx_id != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(MB_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        slot.ptr = static_cast<NoAllocScratch*>(p);
        // the lookup made the context current if it was not yet
        slot.ctx_id = current_context_id(&id) ? id : 0ull;
    }
    *out = slot.ptr;
    return MB_OK;
}

}  // namespace

extern "C" int mb_energy_sum_noalloc(const float* d_ex, const float* d_ey, const float* d_ez,
                                     const float* d_hx, const float* d_hy, const float* d_hz,
                                     const float* d_eps_r, int64_t ncell, double* d_out,
                                     void* cuda_stream) {
    if (!d_ex || !d_ey || !d_ez || !d_hx || !d_hy || !d_hz || !d_out)
        return noalloc_fail(MB_ERR_ARG, "null device pointer");
    if (ncell < 1) return noalloc_fail(MB_ERR_ARG, "ncell must be >= 1");
    if (ncell > kNoAllocMaxCells)
        return noalloc_fail(MB_ERR_ARG, "ncell exceeds the no-allocation limit of 67108864 cells "
                                        "(8192 partial sums of 8192 cells); use mb_energy");
    NoAllocScratch* scratch = nullptr;
    if (int rc = noalloc_scratch(&scratch)) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nparts = (int)((ncell + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock);
    // the flag keeps the last call's value: clear it first
    cudaError_t e = cudaMemsetAsync(&scratch->nonfinite, 0, sizeof(int), s);
    if (e != cudaSuccess) return noalloc_fail(MB_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    k_energy_partial_static<<<nparts, kNoAllocThreads, 0, s>>>(d_ex, d_ey, d_ez, d_hx, d_hy, d_hz,
                                                               d_eps_r, ncell, scratch);
    k_energy_final_static<<<1, 1024, 0, s>>>(scratch, nparts, d_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(MB_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return MB_OK;
}
