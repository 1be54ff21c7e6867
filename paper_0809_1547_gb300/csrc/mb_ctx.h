// Helpers shared by the two host files of the C ABI (mb_api.cu: context,
// materials, probes, read-outs; mb_step.cu: stepping, field copies, tuning).
// Internal to the library.
#pragma once

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mb_host.h"

namespace mbi {

// NVTX range over a host call (seen by profilers that record NVTX; no cost
// otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Allocation-failure injection for tests (mb_debug_fail_alloc): true when
// the next device allocation of a context should fail.
bool inject_alloc_failure();

// Records msg as the context's (and the thread's) last error; returns code.
int fail(mb_ctx* ctx, int code, const std::string& msg);

#define MB_CUDA(ctx, call)                                                                    \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            return mbi::fail((ctx), (e_ == cudaErrorMemoryAllocation) ? MB_ERR_OOM : MB_ERR_CUDA, \
                             std::string(#call) + ": " + cudaGetErrorString(e_));             \
        }                                                                                     \
    } while (0)

// Null check; check_ctx also orders the context's stream after the probe
// launches mb_step may have left on the second stream (mb_step itself and
// the face-energy read use check_ctx_nojoin).
int check_ctx(mb_ctx* c);
int check_ctx_nojoin(mb_ctx* c);
// Device error flag (a bounded wait gave up): MB_ERR_TIMEOUT, flag cleared.
int check_device_error(mb_ctx* c);

// E, H block (6 arrays) and CPML memories of copy p (0: the context's own
// arrays, 1: the single-pass step's second copy).
float* eh_of(const mb_ctx* c, int p);
float* psi_of(const mb_ctx* c, int p, int w);
// Points the step arguments' E, H and CPML memories at copy p.
void point_args_at(mb::StepArgs& a, const mb_ctx* c, int p);

// Device buffers that make up the evolving state (in blob order).
struct StatePart {
    void* ptr;
    size_t bytes;
};
std::vector<StatePart> state_parts(mb_ctx* c);

// Tensor maps of the two-pass TMA launches over the current copy, else nullptr.
const mb::TmaMaps* tma_for(mb_ctx* c, const mb::PassTune& t);

// The probes of one step: point, face and plane DFTs of the fields in a;
// ctr holds the step index of those fields.
void launch_probes(mb_ctx* c, const mb::StepArgs& a, const long long* ctr, cudaStream_t s);
void launch_probes(mb_ctx* c);
bool has_probes(const mb_ctx* c);

// Launches of one step (two passes, or the single-pass step) plus the probes.
int launches_per_step(const mb_ctx* c, bool fused = false);
void drop_graphs(mb_ctx* c);

// Launch shapes chosen per grid shape and CPML depth in this process.
struct TuneSet {
    mb::PassTune h, e, f;
    bool fused;
};
extern std::mutex g_tune_mu;
extern std::map<std::tuple<int, int, int, int>, TuneSet> g_tune_cache;

}  // namespace mbi
