// Host-side structures of the Maxwell–Bloch FDTD library (internal).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "mb_device.cuh"
#include "mb_fdtd.h"

namespace mb {

// exp(i w t) as an FP32 pair (cos, sin): the angle w t is reduced to
// [-pi, pi] in FP64 (w t stays below ~1e6 rad in any run here, so the
// reduction is exact to ~1e-10 rad), then its FP32 sine and cosine are
// taken.  The factor multiplies FP32 field values, so FP32 is its natural
// precision; the FP64 sincos it replaces is slow on this GPU's FP64 pipe.
__device__ __forceinline__ float2 phase_f32(double w, double t) {
    const double two_pi = 6.283185307179586476925;
    const double x = w * t;
    const double r = fma(-two_pi, rint(x * (1.0 / two_pi)), x);
    float s, c;
    sincosf((float)r, &s, &c);
    return make_float2(c, s);
}

struct DevPointProbes {
    int count;
    int nfreq;          // bins per probe (all probes share one count)
    const int64_t* cell;
    const double* omega;   // [count][nfreq]
    double2* acc;          // [count][3][nfreq]
};

// Running DFT of probe p (one block, threads over bins; with k_step > 0 the
// block takes bins k_begin + tid, stepping by k_step) with E_c^{n1} at
// t = n1 dt: acc[p][c][k] += E_c exp(i w_k t) (scaled; times dt E0 on read-out).
__device__ __forceinline__ void point_dft_block(const DevPointProbes& pp, int p, const float* ex,
                                                const float* ey, const float* ez, long long n1,
                                                double dt, int k_begin = 0, int k_step = 0) {
    const double t = (double)n1 * dt;
    const int64_t cell = pp.cell[p];
    const float e[3] = {ex[cell], ey[cell], ez[cell]};
    const int K = pp.nfreq;
    const int T = blockDim.x * blockDim.y * blockDim.z;
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    for (int kk = k_begin + tid; kk < K; kk += (k_step > 0 ? k_step : T)) {
        const float2 w = phase_f32(pp.omega[p * K + kk], t);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double2* acc = pp.acc + ((int64_t)p * 3 + c) * K + kk;
            double2 v = *acc;
            v.x += (double)e[c] * (double)w.x;
            v.y += (double)e[c] * (double)w.y;
            *acc = v;
        }
    }
}

// Face probes: the running DFT sums of each point are kept in FP64 (acc);
// each call adds its terms to FP32 partial sums (acc32), which are added
// into acc and cleared on every kFaceChunk-th call, so the FP64 pipe works
// once per kFaceChunk calls.  A spectrum reads acc + acc32.
constexpr int kFaceChunk = 16;
struct DevFaceProbes {
    int on;
    int stride, every, nfreq, pts_per_block;
    int plane[6];       // plane index along the face normal
    int r0a[6], r0b[6]; // first transverse coordinate along (a, b)
    int na[6], npts[6]; // points along a, total points
    int offset[6];      // first point of each face in acc
    const double* omega;
    double2* acc;       // [point][4][nfreq]: Ea, Eb, Ha, Hb
    float2* acc32;      // the same layout: the sums since the last flush
};

// Whole-plane probe: running DFT of (Ex, Ey, Ez) on every cell of the plane
// z = k, every `every` steps (scaled; times every dt E0 on read-out).
constexpr int kPlaneMaxFreq = 64;
struct DevPlaneProbe {
    int k, every, nfreq;
    const double* omega;   // [nfreq]
    double2* acc;          // [nfreq][3][ny][nx]
};

// Launch shape of one field pass: the 3-D tiled variant (one thread per
// cell, block = (bx, by, bz)) or the z-marching variant (2-D block (bx, by),
// each thread walks kz planes).
constexpr int kVariant3D = 0;
constexpr int kVariantZmarch = 1;
constexpr int kVariantTma = 2;   // TMA-staged z-walk (nx % 16 == 0)
constexpr int kVariantVec = 3;   // z-walk over quads of 4 x-cells, 16-byte accesses (nx % 4 == 0)
struct PassTune {
    int variant;
    dim3 block;
    int kz;
};

// Polls of a bounded mbarrier wait before the kernel gives up (~0.1-1 s).
constexpr int kWaitLimit = 1 << 20;

// Tensor maps of one tile shape (bx, by) for both TMA-staged passes.  E
// pass: H with its -x/-y halo (boxes (bx+4) x (by+1) from (x0-4, y0-1)), E
// and the material byte (bx x by).  H pass: E with its +x/+y halo (boxes
// (bx+4) x (by+1) from (x0, y0)) and H (bx x by).  One plane deep.
struct TmaMaps {
    CUtensorMap hx, hy, hz, ex, ey, ez, mat;   // E pass
    CUtensorMap ebx, eby, ebz, hsx, hsy, hsz;  // H pass
};

// Shared-memory stage of the TMA E pass (each sub-buffer 128-byte aligned).
template <int BX, int BY>
struct TmaLayoutE {
    static constexpr int kHW = (BX + 4) * (BY + 1);
    static constexpr int kEW = BX * BY;
    static constexpr int kHBytes = (kHW * 4 + 127) / 128 * 128;
    static constexpr int kEBytes = (kEW * 4 + 127) / 128 * 128;
    static constexpr int kMBytes = (kEW + 127) / 128 * 128;
    static constexpr int kStage = 3 * kHBytes + 3 * kEBytes + kMBytes;
    static constexpr int kTx = 3 * kHW * 4 + 3 * kEW * 4 + kEW;   // bytes per stage
    // gain-cell J and n1..n3 of two planes (cp.async double buffer)
    static constexpr int kGBytes = 2 * 6 * kEW * 4;
    static constexpr int smem_bytes(int stages) { return stages * kStage + kGBytes + 64 + 128; }
};

// Shared-memory stage of the TMA H pass: E with the +x/+y halo and H of one
// plane; the tile's top stage (plane k1) carries E only.
template <int BX, int BY>
struct TmaLayoutH {
    static constexpr int kEW = (BX + 4) * (BY + 1);
    static constexpr int kHW = BX * BY;
    static constexpr int kEBytes = (kEW * 4 + 127) / 128 * 128;
    static constexpr int kHBytes = (kHW * 4 + 127) / 128 * 128;
    static constexpr int kStage = 3 * kEBytes + 3 * kHBytes;
    static constexpr int kTxE = 3 * kEW * 4;
    static constexpr int kTx = kTxE + 3 * kHW * 4;
    static constexpr int smem_bytes(int stages) { return stages * kStage + 64 + 128; }
};
constexpr int kTmaStages = 3;

bool tma_e_supported(const StepArgs& a);
bool vec_supported(const StepArgs& a);
bool encode_tma(const StepArgs& a, int bx, int by, TmaMaps* out);
// 3-D tensor map over one (nx, ny, nz) array of esize-byte elements with a
// (bw, bh, 1) box, zero fill beyond the array.
bool encode_box(CUtensorMap* m, CUtensorMapDataType dt, const void* base, int esize,
                const DevGrid& g, int bw, int bh);

// Single-pass step (H half-step, Lorentz update, E / population update in
// one launch) reading one copy of E / H / CPML memories and writing the
// other.  Tensor maps of one tile shape (bx, by) over the source copy: E
// with a one-cell halo on every side (boxes (bx+8) x (by+2) from
// (x0-4, y0-1)), H with its -x/-y halo ((bx+4) x (by+1) from (x0-4, y0-1))
// and the material byte (bx x by).
struct TmaFusedMaps {
    CUtensorMap ex, ey, ez, hx, hy, hz, mat;
};
bool fused_tile_supported(int bx, int by);
bool encode_fused(const StepArgs& a, int bx, int by, TmaFusedMaps* out);
void launch_fused_step(const StepArgs& a, const DevPing& d, const PassTune& t,
                       const TmaFusedMaps& maps, cudaStream_t s);

// Grid of the H + gain launch: nH H tiles (tile grid gx x gy x gz) and nG
// gain blocks, each over q consecutive entries of the gain list.
struct HGLayout {
    int gx, gy, gz;
    int nH, nG;
    int q;
};

HGLayout hg_layout(const StepArgs& a, const PassTune& t);
// tma: tensor maps for t's tile shape when t.variant == kVariantTma
void launch_h_pass(const StepArgs& a, const PassTune& t, const TmaMaps* tma, cudaStream_t s);
// tma: tensor maps for t's tile shape when t.variant == kVariantTma
void launch_e_pass(const StepArgs& a, const PassTune& t, const TmaMaps* tma, cudaStream_t s);
void launch_point_dft(const DevPointProbes& pp, const DevFields& f, const long long* ctr,
                      double dt, cudaStream_t s);
void launch_face_dft(const DevFaceProbes& fp, const DevFields& f, const DevGrid& g,
                     const long long* ctr, double dt, cudaStream_t s);
// Batched ensemble, persistent mode: instances advanced together by one
// persistent launch.
// Work items (int4): x = instance, y = kind (0 H tile, 1 gain chunk, 2 E
// tile), z = tile / chunk index.
struct BatchArgs {
    const StepArgs* inst;          // [ninst], device
    const DevPointProbes* probes;  // [ninst], device (count 0: no probe)
    int ninst;
    const int4* items1;            // phase 1: H tiles and gain chunks
    int n1;
    const int4* items2;            // phase 2: E tiles
    int n2;
    const int* tiles;              // [ninst][2]: tile-grid gx, gy of each instance
    int kz, gq;
    unsigned* bar;                 // grid barrier: [0] arrivals, [1] generation
    unsigned long long* tick;      // work-item tickets (zero between launches)
    int* err;
    long long* ctr;                // steps completed by the batch
    int nsteps;
    double dt;
};
constexpr int kBarrierSpinLimit = 1 << 22;   // ~0.3-1 s with 64 ns sleeps
constexpr int kGainPerThread = 2;             // gain cells per thread in a gain block
constexpr int kBatchGainPerThread = 1;        // the same inside the persistent kernel
constexpr int kBatchGainSub = 8;              // gain blocks per work item of the persistent kernel
cudaError_t launch_batch(const BatchArgs& b, dim3 block, int blocks, cudaStream_t s);
// Bounded-wait self-tests: a grid barrier that one phantom block never
// reaches, an mbarrier that is never completed; gave_up counts the blocks
// whose wait ended unfulfilled.
cudaError_t launch_selftest_barrier(unsigned* bar, int blocks, int limit, int* gave_up, cudaStream_t s);
cudaError_t launch_selftest_mbarrier(int limit, int* gave_up, cudaStream_t s);
int batch_blocks_per_sm(dim3 block);

void launch_plane_dft(const DevPlaneProbe& pp, const DevFields& f, const DevGrid& g,
                      const long long* ctr, double dt, cudaStream_t s);
// Energy density of the cells of plane z = k in units of eps0 E0^2 (FP64).
void launch_plane_energy(const DevFields& f, const DevGrid& g, int k, const float* lut_eps,
                         double* out, cudaStream_t s);
void launch_philox(const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, int n, cudaStream_t s);
// out[q] = scale * sum_t slots[q kFluxSlots + t] (slots in order), q < 6.
void launch_flux_sum(const double* slots, double* out, double scale, cudaStream_t s);
// The gain cells (material bit 7) of mat[0, N) in increasing order into
// list: launch_gain_count leaves their number in scratch[gain_list_scratch(N)
// - 2] (scratch holds gain_list_scratch(N) counters), launch_gain_scatter
// then writes the list.
size_t gain_list_scratch(int64_t N);
void launch_gain_count(const uint8_t* mat, int64_t N, uint32_t* scratch, cudaStream_t s);
void launch_gain_scatter(const uint8_t* mat, int64_t N, const uint32_t* scratch, uint32_t* list,
                         cudaStream_t s);
// The material map on the device: the distinct eps_r values into keys
// (kMatKeys entries, kNoKey where unused, filled as a prefix) with the first
// cell of each into first (initialised to kNoKey; flags[0]: a value not
// finite or below 1, flags[1]: more than kMatKeys values), then the material
// bytes from the table put in order of first appearance (launch_mat_ids;
// dense: 1/eps_r per cell into inv_eps and id 0).
constexpr int kMatKeys = 128;
constexpr uint32_t kNoKey = 0xffffffffu;
void launch_mat_keys(const float* eps, int64_t N, uint32_t* keys, uint32_t* first, int* flags,
                     cudaStream_t s);
void launch_mat_ids(const float* eps, const uint8_t* gain, int64_t N, const uint32_t* keys, int n,
                    bool dense, bool gain_on, uint8_t* mat, float* inv_eps, cudaStream_t s);
void launch_energy(const DevFields& f, int64_t ncell, const float* lut_eps, double* partial,
                   int nparts, int* nonfinite, double* out, cudaStream_t s);

// Message returned by mb_last_error(NULL) on this thread.
void set_thread_error(const std::string& msg);

// Tensor maps of the context's TMA E pass for tuning t (nullptr if t is not
// a TMA tuning or the maps cannot be encoded).
const TmaMaps* tma_maps(mb_ctx* c, const PassTune& t);

// Enqueue one full step exactly as mb_step runs it, without a graph (the two
// passes with the context's tuning, then the probes); advances the count.
cudaError_t enqueue_step(mb_ctx* c);

// Brings the state back into the context's own copy (d_fields, d_psi) and
// switches the single-pass step off (returning whether it was on), so that
// every later step runs in place; restore_single_pass undoes the switch.
bool hold_in_place(mb_ctx* c);
void restore_single_pass(mb_ctx* c, bool on);
// Orders the context's stream after every probe launch that mb_step left
// running on the second stream (event waits only; never blocks the host).
void join_probes(mb_ctx* c);

// d/dW_p of the reduced population propagator (g, G, mk of DevGain).
void gain_pump_derivative(const mb_ctx* c, float dg[3], float dG[3][3], float dmk[3]);

// Whole evolving state of a context as one device blob (for device-side
// snapshots: autotuning, adjoint checkpoints).
size_t state_device_bytes(mb_ctx* c);
int state_snapshot(mb_ctx* c, void* d_dst);          // device -> device, on c's stream
int state_restore(mb_ctx* c, const void* d_src);     // device -> device, on c's stream

// Physical constants (SI, CODATA 2018).
constexpr double kC0 = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kHbar = 1.054571817e-34;
constexpr double kQe = 1.602176634e-19;
constexpr double kPi = 3.14159265358979323846;

struct PointProbeHost {
    int64_t cell;
    int nfreq;
    std::vector<double> lam, omega;
};

}  // namespace mb

struct mb_ctx {
    int nx = 0, ny = 0, nz = 0;
    int64_t ncell = 0;
    // z-window.  A context may hold one z-slab of a grid split along z
    // (mb_create_slab): local plane k is plane k + kz0 of the whole grid of
    // gnz planes; planes [own_lo, own_hi) are the slab's own, the others (at
    // most one below and one above) are ghost planes that receive the
    // neighbouring slabs' boundary planes before every step.  A whole grid
    // has gnz = nz, kz0 = 0, own_lo = 0, own_hi = nz.
    bool slab = false;
    int gnz = 0, kz0 = 0, own_lo = 0, own_hi = 0;
    double dx = 0, dt = 0;
    mb_params p{};
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    // scales between SI and the device units
    double E0 = 0, eta0 = 0, S = 0;

    // device memory
    float* d_fields = nullptr;         // 15 arrays of ncell floats
    uint8_t* d_mat = nullptr;
    float* d_inv_eps = nullptr;        // dense 1/eps_r (only when > 128 materials)
    float* d_lut = nullptr;            // [0..127]: 1/eps_r, [128..255]: eps_r
    float* d_psi[3] = {nullptr, nullptr, nullptr};
    size_t psi_elems[3] = {0, 0, 0};
    float* d_coef = nullptr;           // CPML tables
    uint32_t* d_glist = nullptr;       // gain cells, increasing order
    uint32_t glist_count = 0;
    size_t glist_capacity = 0;
    uint32_t* d_glist_scratch = nullptr;   // per-chunk counters of the list build
    size_t glist_scratch_n = 0;
    // step counters: [0] steps completed, [1] finished blocks of the current
    // launch, [2 + q] the step count when copy q was last written by the
    // single-pass step (the probes of that copy sample it)
    long long* d_ctr = nullptr;
    double* d_flux = nullptr;          // 6 faces x kFluxSlots accumulators
    double* d_flux_out = nullptr;      // the 6 face energies in joules (read-back staging)
    double* d_partial = nullptr;       // energy partial sums
    double* d_energy = nullptr;
    int* d_nonfinite = nullptr;
    int n_partial = 0;

    // point probes
    std::vector<mb::PointProbeHost> probes;
    int64_t* d_probe_cell = nullptr;
    double* d_probe_omega = nullptr;
    double2* d_probe_acc = nullptr;
    int probe_nfreq = 0;

    // whole-plane probes (mode maps)
    std::vector<mb::DevPlaneProbe> planes;   // device pointers owned here
    std::vector<std::vector<double>> plane_lam;

    // face probes
    mb::DevFaceProbes face{};
    std::vector<double> face_lam;
    double* d_face_omega = nullptr;
    double2* d_face_acc = nullptr;
    float2* d_face_acc32 = nullptr;
    int64_t face_points = 0;

    // material
    bool have_material = false;
    bool dense_eps = false;
    // mb_set_material's device scratch: the uploaded eps_r map and gain mask
    // (5 bytes per cell), the table of distinct values and two flags
    uint8_t* d_upload = nullptr;
    size_t upload_bytes = 0;
    uint32_t* d_keys = nullptr;
    size_t keys_bytes = 0;
    std::vector<float> h_lut_eps;      // eps_r per material id
    int n_lut = 128;                   // entries of the table (128: unknown or dense)
    float h_lut_ie[2] = {1.0f, 1.0f};  // 1/eps_r of ids 0 and 1
    double N_a = 0, W_p = 0;
    uint64_t seed = 0;

    // per-step arguments
    mb::StepArgs args{};
    mb::DevSource src{};
    float* d_src_wave = nullptr;       // tabulated source current
    int* d_err = nullptr;              // device error flag (bounded waits)
    std::map<std::tuple<int, int, int>, mb::TmaMaps> tma_maps;   // per TMA tile shape and copy
    mb::PassTune tune_h{mb::kVariantZmarch, dim3(32, 8, 1), 16};
    mb::PassTune tune_e{mb::kVariantZmarch, dim3(32, 4, 1), 16};

    // single-pass step: each step reads one copy of E, H and the CPML
    // memories and writes the other; `parity` says which copy holds the
    // current state (0: d_fields / d_psi, 1: d_fields2 / d_psi2) and args
    // always points at it.  P, J and the populations have one copy.
    bool use_fused = false;
    mb::PassTune tune_f{mb::kVariantTma, dim3(32, 8, 1), 32};
    float* d_fields2 = nullptr;        // second copy of E, H (6 arrays)
    float* d_psi2[3] = {nullptr, nullptr, nullptr};
    int parity = 0;
    std::map<std::pair<int, int>, std::pair<mb::TmaFusedMaps, mb::TmaFusedMaps>> fused_maps;

    // stepping
    int64_t n = 0;
    int64_t launches = 0;
    // the single-pass step's probes run on a second stream, concurrently
    // with the next step (fork / join events of a captured chunk)
    cudaStream_t aux_stream = nullptr;
    std::vector<cudaEvent_t> fork_ev, join_ev;
    // Probes of single steps (mb_step's remainder after whole chunks) are
    // left running on the second stream: probe_pending[q] while the launch
    // that reads copy q may still run (probe_done[q] recorded after it,
    // probe_fork[q] orders it after its step).  The next step writing copy q
    // waits for it; every other call joins first (join_probes).
    bool probe_pending[2] = {false, false};
    cudaEvent_t probe_fork[2] = {nullptr, nullptr};
    cudaEvent_t probe_done[2] = {nullptr, nullptr};
    // per parity of the starting copy (the pointers baked into a graph)
    cudaGraphExec_t graph_chunk[2] = {nullptr, nullptr};
    cudaGraphExec_t graph_one[2] = {nullptr, nullptr};
    bool graph_fused = false;          // mode the graphs were captured in
    int graph_chunk_steps = 16;        // even: a chunk returns to its starting copy

    std::string err;
    size_t dev_bytes = 0;
};
