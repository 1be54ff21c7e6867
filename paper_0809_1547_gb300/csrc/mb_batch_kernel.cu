// The batched ensemble's persistent kernel: every member's H tiles, gain
// chunks and E tiles in one cooperative launch per call, with bounded grid
// barriers between the phases.
#include "mb_host.h"
#include "mb_tiles.cuh"
#include "mb_tma.cuh"

namespace mb {

// ---------------------------------------------------- batched ensemble
// Grid-wide barrier of a co-resident (cooperative) grid, with a bounded
// wait: false when the other blocks did not all arrive within `limit` polls.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int limit = kBarrierSpinLimit) {
    __shared__ int ok_s;
    __syncthreads();
    if (linear_tid() == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            for (int it = 0; *gen == g; ++it) {
                if (it > limit) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Arguments of the item's instance, copied into shared memory: global
// stores cannot alias them there, so the field pointers need not stay in
// registers or be reloaded after every store.  One copy per item kind
// (TAG); an item of the instance whose arguments the copy already holds
// (a block's consecutive items are often tiles of one instance) skips the
// copy.  The arguments do not change during a launch.
__shared__ int staged_inst[3];   // instance held by each copy, -1: none

__device__ __forceinline__ void staged_reset() {
    if (linear_tid() < 3) staged_inst[linear_tid()] = -1;
    __syncthreads();
}

template <int TAG>
__device__ __forceinline__ const StepArgs& stage_args(const StepArgs* inst, int p) {
    static_assert(sizeof(StepArgs) % 8 == 0, "StepArgs is copied in 8-byte words");
    __shared__ StepArgs sa;
    if (staged_inst[TAG] != p) {   // uniform: read after the caller's barrier
        const unsigned long long* s8 = reinterpret_cast<const unsigned long long*>(inst + p);
        unsigned long long* d8 = reinterpret_cast<unsigned long long*>(&sa);
        const int T = blockDim.x * blockDim.y * blockDim.z;
        for (int t = linear_tid(); t < (int)(sizeof(StepArgs) / 8); t += T) d8[t] = s8[t];
        __syncthreads();   // every thread has read staged_inst before it changes
        if (linear_tid() == 0) staged_inst[TAG] = p;
        __syncthreads();
    }
    return sa;
}

// Work items of the persistent kernel, each its own (not inlined) function
// so that the register allocation of one phase does not burden the others.
// The caller has synchronised the block since the previous item.
__device__ __noinline__ void batch_probe_item(const BatchArgs& B, int p, long long n) {
    const StepArgs& a = B.inst[p];
    for (int q = 0; q < B.probes[p].count; ++q)
        point_dft_block(B.probes[p], q, a.f.ex, a.f.ey, a.f.ez, n, B.dt);
}

__device__ __noinline__ void batch_h_item(const BatchArgs& B, int4 it) {
    const StepArgs& a = stage_args<0>(B.inst, it.x);
    const int gx = B.tiles[2 * it.x], gy = B.tiles[2 * it.x + 1];
    h_tile_zmarch(a, it.z % gx, (it.z / gx) % gy, it.z / (gx * gy), B.kz);
}

// kBatchGainSub consecutive blocks of B.gq gain-list entries (the block's
// threads one entry each, block after block): fewer, larger items than one
// block of entries each, so the ticket and the barriers around an item are
// paid less often.
__device__ __noinline__ void batch_gain_item(const BatchArgs& B, int4 it, long long n) {
    const StepArgs& a = stage_args<1>(B.inst, it.x);
#pragma unroll 1
    for (int s = 0; s < kBatchGainSub; ++s)
        gain_block<kBatchGainPerThread>(a, (unsigned)it.z * kBatchGainSub + s, B.gq, n);
}

__device__ __noinline__ void batch_e_item(const BatchArgs& B, int4 it, long long n, unsigned slot) {
    const StepArgs& a = stage_args<2>(B.inst, it.x);
    const int gx = B.tiles[2 * it.x], gy = B.tiles[2 * it.x + 1];
    e_tile_zmarch(a, it.z % gx, (it.z / gx) % gy, it.z / (gx * gy), B.kz, n, slot);
}

// Next work item of this block in the current phase: tickets are drawn from
// one counter; tickets [base, base + n) are the phase's items, and every
// block draws exactly one ticket past them before it leaves the phase, so the
// next phase starts at base + n + gridDim.x.  Returns -1 when the phase is
// exhausted.
__device__ __forceinline__ int next_item(unsigned long long* tick, unsigned long long base, int n) {
    __shared__ int item_s;
    __syncthreads();   // the previous item is finished by every thread
    if (linear_tid() == 0) {
        const unsigned long long t = atomicAdd(tick, 1ull) - base;
        item_s = t < (unsigned long long)n ? (int)t : -1;
    }
    __syncthreads();
    return item_s;
}

// n steps of every instance in one launch.  Per step: phase 1 = the point
// probes of the previous step (they read E only) + all instances' H tiles
// and gain chunks; barrier; phase 2 = all E tiles; barrier.  Blocks draw
// items from a shared counter in list order (which keeps neighbouring tiles
// together for L2 reuse), so grids of uneven size and cost balance.  A barrier that times out sets the error
// flag and the block leaves; the other blocks then time out at their next
// barrier, so the launch always ends.
__global__ void __launch_bounds__(256, 4) k_batch(const __grid_constant__ BatchArgs B) {
    staged_reset();
    const unsigned nb = gridDim.x;
    const long long n0 = B.ctr[0];
    unsigned long long base = 0;
    for (int s = 0; s < B.nsteps; ++s) {
        const long long n = n0 + s;
        if (s > 0)
            for (int p = blockIdx.x; p < B.ninst; p += nb) batch_probe_item(B, p, n);
        for (int w; (w = next_item(B.tick, base, B.n1)) >= 0;) {
            const int4 it = B.items1[w];
            if (it.y == 0) batch_h_item(B, it);
            else batch_gain_item(B, it, n);
        }
        base += (unsigned long long)B.n1 + nb;
        if (!grid_barrier(B.bar, nb)) {
            if (linear_tid() == 0) atomicOr(B.err, 1);
            return;
        }
        for (int w; (w = next_item(B.tick, base, B.n2)) >= 0;)
            batch_e_item(B, B.items2[w], n, (unsigned)w * 7u + (linear_tid() >> 5));
        base += (unsigned long long)B.n2 + nb;
        if (!grid_barrier(B.bar, nb)) {
            if (linear_tid() == 0) atomicOr(B.err, 1);
            return;
        }
    }
    const long long n_end = n0 + B.nsteps;
    for (int p = blockIdx.x; p < B.ninst; p += nb) batch_probe_item(B, p, n_end);
    if (blockIdx.x == 0) {
        // every block read n0 before the first barrier and drew its last
        // ticket before the last one; nsteps >= 1
        for (int p = linear_tid(); p < B.ninst; p += blockDim.x * blockDim.y) B.inst[p].step_ctr[0] = n_end;
        if (linear_tid() == 0) {
            B.ctr[0] = n_end;
            *B.tick = 0ull;
        }
    }
}

int batch_blocks_per_sm(dim3 block) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch, block.x * block.y * block.z, 0) !=
        cudaSuccess)
        return 0;
    return n;
}

cudaError_t launch_batch(const BatchArgs& b, dim3 block, int blocks, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks, 1, 1);
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;   // all blocks co-resident: the barrier is safe
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch, b);
}

// ------------------------------------------------- bounded-wait self-test
// The waits of the batched and TMA kernels must end by themselves when the
// awaited event never comes.  These kernels run the same wait code against
// events that cannot happen and record whether it gave up.
// Grid barrier counting one block more than the grid holds.
__global__ void k_selftest_barrier(unsigned* bar, int limit, int* gave_up) {
    if (!grid_barrier(bar, gridDim.x + 1, limit) && linear_tid() == 0) atomicAdd(gave_up, 1);
}

// An mbarrier that expects one arrival that never comes.
__global__ void k_selftest_mbarrier(int limit, int* gave_up) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const bool done = mbar_wait_bounded(&bar, 0, limit);
    if (!done && threadIdx.x == 0) atomicAdd(gave_up, 1);
}

cudaError_t launch_selftest_barrier(unsigned* bar, int blocks, int limit, int* gave_up, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks, 1, 1);
    cfg.blockDim = dim3(64, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_selftest_barrier, bar, limit, gave_up);
}

cudaError_t launch_selftest_mbarrier(int limit, int* gave_up, cudaStream_t s) {
    k_selftest_mbarrier<<<1, 32, 0, s>>>(limit, gave_up);
    return cudaGetLastError();
}

}  // namespace mb
