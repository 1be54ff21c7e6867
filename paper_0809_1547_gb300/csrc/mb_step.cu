// C ABI of the Maxwell–Bloch FDTD library, stepping: the two copies of E, H
// and the CPML memories the single-pass step alternates between, CUDA-graph
// capture of step chunks (with the probes of a single-pass step overlapped
// with the next step on a second stream), direct timed steps, the launch-
// shape autotuner and the tuning calls.
#include "mb_ctx.h"

#include <algorithm>
#include <cstring>
#include <mutex>

namespace mbi {

// ---- single-pass step: the two copies of E, H and the CPML memories

// Step arguments over copy p (P, J, populations, material, tables and
// counters shared with the context's own arguments).
mb::StepArgs view_of(const mb_ctx* c, int p) {
    mb::StepArgs b = c->args;
    point_args_at(b, c, p);
    return b;
}

// Destination of a single-pass step writing copy q (viewed by a).
mb::DevPing ping_of(const mb_ctx* c, const mb::StepArgs& a, int q) {
    return mb::DevPing{a.f.ex, a.f.ey, a.f.ez, a.f.hx, a.f.hy, a.f.hz,
                       mb::PsiOut{a.pml.psx, a.pml.psy, a.pml.psz}, c->d_ctr + 2 + q};
}

// Allocates the second copy on first use.
int ensure_second_copy(mb_ctx* c) {
    if (c->d_fields2) return MB_OK;
    const size_t fb = sizeof(float) * 6 * (size_t)c->ncell;
    cudaError_t e = inject_alloc_failure() ? cudaErrorMemoryAllocation
                                           : cudaMalloc((void**)&c->d_fields2, fb);
    for (int w = 0; w < 3 && e == cudaSuccess; ++w)
        if (c->psi_elems[w]) e = cudaMalloc((void**)&c->d_psi2[w], sizeof(float) * c->psi_elems[w]);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->d_fields2);
        for (int w = 0; w < 3; ++w) cudaFree(c->d_psi2[w]);
        c->d_fields2 = nullptr;
        c->d_psi2[0] = c->d_psi2[1] = c->d_psi2[2] = nullptr;
        return fail(c, MB_ERR_OOM, "cudaMalloc of the single-pass step's second field copy failed");
    }
    c->dev_bytes += fb;
    for (int w = 0; w < 3; ++w) c->dev_bytes += sizeof(float) * c->psi_elems[w];
    return MB_OK;
}

// Tensor maps of the single-pass step for tile shape t reading (copy 0,
// copy 1), encoded once per shape; nullptr if unsupported.
const std::pair<mb::TmaFusedMaps, mb::TmaFusedMaps>* fused_maps_for(mb_ctx* c, const mb::PassTune& t) {
    if (!c->d_fields2) return nullptr;
    const auto key = std::make_pair((int)t.block.x, (int)t.block.y);
    auto it = c->fused_maps.find(key);
    if (it != c->fused_maps.end()) return &it->second;
    std::pair<mb::TmaFusedMaps, mb::TmaFusedMaps> m;
    if (!mb::encode_fused(view_of(c, 0), t.block.x, t.block.y, &m.first) ||
        !mb::encode_fused(view_of(c, 1), t.block.x, t.block.y, &m.second))
        return nullptr;
    return &(c->fused_maps[key] = m);
}

// Events for a captured chunk of `steps` single-pass steps (created once).
void ensure_events(mb_ctx* c, int steps) {
    while ((int)c->fork_ev.size() < steps) {
        cudaEvent_t a = nullptr, b = nullptr;
        cudaEventCreateWithFlags(&a, cudaEventDisableTiming);
        cudaEventCreateWithFlags(&b, cudaEventDisableTiming);
        c->fork_ev.push_back(a);
        c->join_ev.push_back(b);
    }
}

// Is the single-pass step usable now (second copy allocated, maps encoded)?
// Falls back to the two passes when not.
bool fused_ready(mb_ctx* c) {
    if (!c->use_fused) return false;
    if (ensure_second_copy(c) != MB_OK || !fused_maps_for(c, c->tune_f)) {
        c->err.clear();
        c->use_fused = false;
        return false;
    }
    return true;
}

// Captures `steps` steps starting from copy p: single-pass steps (each
// flipping the copy) or two-pass steps in place.
int capture_steps(mb_ctx* c, int steps, int p, bool fused, cudaGraphExec_t* out) {
    cudaGraph_t graph = nullptr;
    const std::pair<mb::TmaFusedMaps, mb::TmaFusedMaps>* fm = fused ? fused_maps_for(c, c->tune_f) : nullptr;
    if (fused && !fm) return fail(c, MB_ERR_STATE, "single-pass step maps unavailable");
    const int saved = c->parity;
    c->parity = p;   // two-pass graphs run on copy p
    point_args_at(c->args, c, p);
    const mb::TmaMaps* mh = fused ? nullptr : tma_for(c, c->tune_h);
    const mb::TmaMaps* me = fused ? nullptr : tma_for(c, c->tune_e);
    // Single-pass steps: the probes of step s read only the copy it wrote,
    // which step s + 1 only reads, so they run on the second stream beside
    // step s + 1; step s + 2 (which rewrites that copy) waits for them, and
    // the chunk ends with the second stream joined.
    const bool fork = fused && has_probes(c) && c->aux_stream;
    if (fork) ensure_events(c, steps);
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int s = 0; s < steps; ++s) {
            if (fused) {
                const mb::StepArgs in = view_of(c, p), out = view_of(c, 1 - p);
                if (fork && s >= 2) cudaStreamWaitEvent(c->stream, c->join_ev[s - 2], 0);
                mb::launch_fused_step(in, ping_of(c, out, 1 - p), c->tune_f, p ? fm->second : fm->first,
                                      c->stream);
                if (fork) {
                    cudaEventRecord(c->fork_ev[s], c->stream);
                    cudaStreamWaitEvent(c->aux_stream, c->fork_ev[s], 0);
                    launch_probes(c, out, c->d_ctr + 2 + (1 - p), c->aux_stream);
                    cudaEventRecord(c->join_ev[s], c->aux_stream);
                } else {
                    launch_probes(c, out, c->d_ctr + 2 + (1 - p), c->stream);
                }
                p = 1 - p;
            } else {
                mb::launch_h_pass(c->args, c->tune_h, mh, c->stream);
                mb::launch_e_pass(c->args, c->tune_e, me, c->stream);
                launch_probes(c);
            }
        }
        if (fork) cudaStreamWaitEvent(c->stream, c->join_ev[steps - 1], 0);
        e = cudaStreamEndCapture(c->stream, &graph);
    }
    c->parity = saved;
    point_args_at(c->args, c, saved);
    if (e != cudaSuccess) return fail(c, MB_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(c, MB_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return MB_OK;
}

// The chunk and / or single-step graph starting from copy p in the current
// mode (captured on first use; graphs of the other mode are dropped).
int step_graphs(mb_ctx* c, int p, bool fused, bool chunk, bool one) {
    if (c->graph_fused != fused) {
        drop_graphs(c);
        c->graph_fused = fused;
    }
    int rc = MB_OK;
    if (chunk && !c->graph_chunk[p] &&
        (rc = capture_steps(c, c->graph_chunk_steps, p, fused, &c->graph_chunk[p])))
        return rc;
    if (one && !c->graph_one[p] && (rc = capture_steps(c, 1, p, fused, &c->graph_one[p]))) return rc;
    return MB_OK;
}

// Makes copy p the current one.
void set_parity(mb_ctx* c, int p) {
    c->parity = p;
    point_args_at(c->args, c, p);
}

}  // namespace mbi

using namespace mbi;

bool mb::hold_in_place(mb_ctx* c) {
    const bool on = c->use_fused;
    if (c->parity) {
        const size_t N = (size_t)c->ncell;
        cudaMemcpyAsync(c->d_fields, c->d_fields2, sizeof(float) * 6 * N, cudaMemcpyDeviceToDevice, c->stream);
        for (int w = 0; w < 3; ++w)
            if (c->psi_elems[w])
                cudaMemcpyAsync(c->d_psi[w], c->d_psi2[w], sizeof(float) * c->psi_elems[w],
                                cudaMemcpyDeviceToDevice, c->stream);
        set_parity(c, 0);
    }
    c->use_fused = false;
    return on;
}

void mb::restore_single_pass(mb_ctx* c, bool on) { c->use_fused = on; }

void mb::join_probes(mb_ctx* c) {
    for (int q = 0; q < 2; ++q)
        if (c->probe_pending[q]) {
            cudaStreamWaitEvent(c->stream, c->probe_done[q], 0);
            c->probe_pending[q] = false;
        }
}

namespace mbi {

// One single-pass step from copy p outside a graph, its probes left running
// on the second stream: the step waits for the probes still reading the copy
// it overwrites (those of the step before last), and its own probes read the
// copy it writes, which the next step only reads.
int single_step_deferred(mb_ctx* c, int p) {
    for (int q = 0; q < 2; ++q) {
        if (!c->probe_fork[q]) MB_CUDA(c, cudaEventCreateWithFlags(&c->probe_fork[q], cudaEventDisableTiming));
        if (!c->probe_done[q]) MB_CUDA(c, cudaEventCreateWithFlags(&c->probe_done[q], cudaEventDisableTiming));
    }
    const int q = 1 - p;
    const std::pair<mb::TmaFusedMaps, mb::TmaFusedMaps>* fm = fused_maps_for(c, c->tune_f);
    if (!fm) return fail(c, MB_ERR_STATE, "single-pass step maps unavailable");
    if (c->probe_pending[q]) {
        MB_CUDA(c, cudaStreamWaitEvent(c->stream, c->probe_done[q], 0));
        c->probe_pending[q] = false;
    }
    const mb::StepArgs in = view_of(c, p), out = view_of(c, q);
    mb::launch_fused_step(in, ping_of(c, out, q), c->tune_f, p ? fm->second : fm->first, c->stream);
    MB_CUDA(c, cudaEventRecord(c->probe_fork[q], c->stream));
    MB_CUDA(c, cudaStreamWaitEvent(c->aux_stream, c->probe_fork[q], 0));
    launch_probes(c, out, c->d_ctr + 2 + q, c->aux_stream);
    MB_CUDA(c, cudaEventRecord(c->probe_done[q], c->aux_stream));
    c->probe_pending[q] = true;
    return MB_OK;
}

}  // namespace mbi

cudaError_t mb::enqueue_step(mb_ctx* c) {
    mb::launch_h_pass(c->args, c->tune_h, tma_for(c, c->tune_h), c->stream);
    mb::launch_e_pass(c->args, c->tune_e, tma_for(c, c->tune_e), c->stream);
    launch_probes(c);
    c->n += 1;
    c->launches += launches_per_step(c);
    return cudaGetLastError();
}

extern "C" {

int mb_step(mb_ctx* c, int n) {
    // probes of earlier single steps may keep running beside these steps
    if (int rc = check_ctx_nojoin(c)) return rc;
    NvtxRange range("mb_step");
    if (n < 0) return fail(c, MB_ERR_ARG, "negative step count");
    if (n == 0) return MB_OK;
    const bool fused = fused_ready(c);
    // single-pass steps outside whole chunks leave their probes on the second stream
    const bool defer = fused && has_probes(c) && c->aux_stream;
    int p = c->parity;
    const int chunks = n / c->graph_chunk_steps, rem = n % c->graph_chunk_steps;
    if (chunks > 0 || n >= 2 || !fused) mb::join_probes(c);
    // a call of several steps also prepares the chunk graphs that later calls
    // replay (from either copy for the single-pass step), so their capture
    // falls in a warm-up call rather than in a timed one
    if (n >= 2) {
        if (int rc = step_graphs(c, fused ? 1 - p : p, fused, true, false)) return rc;
    }
    if (chunks > 0 || n >= 2) {
        if (int rc = step_graphs(c, p, fused, true, false)) return rc;
    }
    for (int q = 0; q < chunks; ++q) MB_CUDA(c, cudaGraphLaunch(c->graph_chunk[p], c->stream));
    for (int q = 0; q < rem; ++q) {
        if (defer) {
            if (int rc = single_step_deferred(c, p)) return rc;
        } else {
            if (int rc = step_graphs(c, p, fused, false, true)) return rc;
            MB_CUDA(c, cudaGraphLaunch(c->graph_one[p], c->stream));
        }
        if (fused) p = 1 - p;
    }
    MB_CUDA(c, cudaGetLastError());
    set_parity(c, p);
    c->n += n;
    c->launches += (int64_t)n * launches_per_step(c, fused);
    return MB_OK;
}

int mb_step_timed(mb_ctx* c, int n, double* ms_out) {
    if (int rc = check_ctx(c)) return rc;
    NvtxRange range("mb_step_timed");
    if (n < 0) return fail(c, MB_ERR_ARG, "negative step count");
    if (n == 0) return MB_OK;
    // 5 events per step: before H, after H, after E, after point DFT, after face DFT
    std::vector<cudaEvent_t> ev((size_t)5 * n);
    for (auto& e : ev) {
        cudaError_t ce = cudaEventCreate(&e);
        if (ce != cudaSuccess) {
            for (auto& x : ev)
                if (x) cudaEventDestroy(x);
            return fail(c, MB_ERR_CUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(ce));
        }
    }
    mb::DevPointProbes pp{(int)c->probes.size(), c->probe_nfreq, c->d_probe_cell,
                          c->d_probe_omega, c->d_probe_acc};
    const bool fused = fused_ready(c);
    const std::pair<mb::TmaFusedMaps, mb::TmaFusedMaps>* fm = fused ? fused_maps_for(c, c->tune_f) : nullptr;
    int p = c->parity;
    for (int s = 0; s < n; ++s) {
        cudaEvent_t* e = &ev[(size_t)5 * s];
        // a single-pass step reads copy p and writes the other one
        const mb::StepArgs in = view_of(c, p);
        const mb::StepArgs out = fused ? view_of(c, 1 - p) : in;
        cudaEventRecord(e[0], c->stream);
        if (fused) {
            mb::launch_fused_step(in, ping_of(c, out, 1 - p), c->tune_f, p ? fm->second : fm->first,
                                  c->stream);
            cudaEventRecord(e[1], c->stream);
            p = 1 - p;
        } else {
            mb::launch_h_pass(c->args, c->tune_h, tma_for(c, c->tune_h), c->stream);
            cudaEventRecord(e[1], c->stream);
            mb::launch_e_pass(c->args, c->tune_e, tma_for(c, c->tune_e), c->stream);
        }
        cudaEventRecord(e[2], c->stream);
        const long long* ctr = fused ? c->d_ctr + 2 + p : c->d_ctr;   // p: the copy just written
        mb::launch_point_dft(pp, out.f, ctr, c->dt, c->stream);
        cudaEventRecord(e[3], c->stream);
        mb::launch_face_dft(c->face, out.f, out.g, ctr, c->dt, c->stream);
        for (const mb::DevPlaneProbe& q : c->planes) mb::launch_plane_dft(q, out.f, out.g, ctr, c->dt, c->stream);
        cudaEventRecord(e[4], c->stream);
    }
    cudaError_t le = cudaGetLastError();
    cudaError_t se = cudaStreamSynchronize(c->stream);
    double acc[4] = {0, 0, 0, 0};
    for (int s = 0; s < n && le == cudaSuccess && se == cudaSuccess; ++s) {
        cudaEvent_t* e = &ev[(size_t)5 * s];
        for (int q = 0; q < 4; ++q) {
            float ms = 0;
            cudaEventElapsedTime(&ms, e[q], e[q + 1]);
            acc[q] += ms;
        }
    }
    for (auto& x : ev) cudaEventDestroy(x);
    set_parity(c, p);
    if (le != cudaSuccess) return fail(c, MB_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(le));
    if (se != cudaSuccess) return fail(c, MB_ERR_CUDA, std::string("sync: ") + cudaGetErrorString(se));
    if (ms_out)
        for (int q = 0; q < 4; ++q) ms_out[q] += acc[q];
    c->n += n;
    c->launches += (int64_t)n * launches_per_step(c, fused);
    return check_device_error(c);
}

int mb_autotune(mb_ctx* c) {
    if (int rc = check_ctx(c)) return rc;
    NvtxRange range("mb_autotune");
    auto parts = state_parts(c);
    size_t total = 0;
    for (auto& p : parts) total += p.bytes;
    char* backup = nullptr;
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    MB_CUDA(c, cudaMalloc((void**)&backup, total));
    {
        char* o = backup;
        for (auto& p : parts) {
            cudaMemcpyAsync(o, p.ptr, p.bytes, cudaMemcpyDeviceToDevice, c->stream);
            o += p.bytes;
        }
    }
    std::vector<mb::PassTune> cands;
    for (dim3 b : {dim3(32, 4, 2), dim3(32, 8, 1), dim3(64, 4, 1), dim3(32, 2, 4), dim3(128, 2, 1),
                   dim3(32, 4, 4), dim3(64, 2, 2)})
        cands.push_back({mb::kVariant3D, b, 1});
    for (dim3 b : {dim3(32, 4, 1), dim3(32, 8, 1), dim3(64, 4, 1), dim3(64, 2, 1), dim3(128, 2, 1),
                   dim3(32, 16, 1), dim3(64, 8, 1), dim3(128, 4, 1), dim3(256, 1, 1)})
        for (int kz : {4, 8, 16, 32}) cands.push_back({mb::kVariantZmarch, b, kz});
    if (mb::vec_supported(c->args))
        for (dim3 b : {dim3(32, 2, 1), dim3(32, 4, 1), dim3(32, 8, 1), dim3(64, 2, 1), dim3(64, 4, 1),
                       dim3(128, 2, 1)})
            for (int kz : {4, 8, 16, 32}) cands.push_back({mb::kVariantVec, b, kz});
    if (mb::tma_e_supported(c->args))
        for (dim3 b : {dim3(32, 4, 1), dim3(32, 8, 1), dim3(64, 4, 1), dim3(64, 8, 1), dim3(128, 2, 1),
                       dim3(128, 4, 1)})
            for (int kz : {8, 16, 32, 64}) cands.push_back({mb::kVariantTma, b, kz});
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_h = 1e30f, best_e = 1e30f;
    mb::PassTune bh = c->tune_h, be = c->tune_e;
    const int reps = c->ncell > 4000000 ? 2 : 6;
    for (const mb::PassTune& t : cands) {
        if (t.variant != mb::kVariant3D && t.kz > 2 * c->nz) continue;
        if (t.variant == mb::kVariantTma && !tma_for(c, t)) continue;
        for (int pass = 0; pass < 2; ++pass) {
            if (pass == 0) mb::launch_h_pass(c->args, t, tma_for(c, t), c->stream);
            else mb::launch_e_pass(c->args, t, tma_for(c, t), c->stream);
            cudaEventRecord(e0, c->stream);
            for (int r = 0; r < reps; ++r) {
                if (pass == 0) mb::launch_h_pass(c->args, t, tma_for(c, t), c->stream);
                else mb::launch_e_pass(c->args, t, tma_for(c, t), c->stream);
            }
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (pass == 0 && ms < best_h) { best_h = ms; bh = t; }
            if (pass == 1 && ms < best_e) { best_e = ms; be = t; }
        }
    }
    // the single-pass step against the best pair of passes
    mb::PassTune bf = c->tune_f;
    float best_f = 1e30f;
    if (mb::tma_e_supported(c->args) && ensure_second_copy(c) == MB_OK) {
        // current copy -> other copy, repeated (the other copy is scratch)
        const mb::StepArgs other = view_of(c, 1 - c->parity);
        const mb::DevPing dst = ping_of(c, other, 1 - c->parity);
        // ms per launch of candidate t over n launches (after one untimed)
        auto time_fused = [&](const mb::PassTune& t, int n) -> float {
            const auto* fm = fused_maps_for(c, t);
            if (!fm) return 1e30f;
            const mb::TmaFusedMaps& m = c->parity ? fm->second : fm->first;
            mb::launch_fused_step(c->args, dst, t, m, c->stream);
            cudaEventRecord(e0, c->stream);
            for (int r = 0; r < n; ++r) mb::launch_fused_step(c->args, dst, t, m, c->stream);
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            return ms / n;
        };
        std::vector<std::pair<float, mb::PassTune>> tf;
        for (dim3 b : {dim3(32, 4, 1), dim3(32, 8, 1), dim3(64, 4, 1), dim3(64, 8, 1)})
            for (int kz : {8, 12, 16, 20, 24, 32, 48, 64}) {
                const mb::PassTune t{mb::kVariantTma, b, kz};
                if (kz > 2 * c->nz) continue;
                tf.push_back({time_fused(t, reps), t});
            }
        // the three fastest again, longer and twice interleaved (neighbouring
        // shapes often time within a percent of each other): the best minimum
        std::sort(tf.begin(), tf.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
        if (tf.size() > 3) tf.resize(3);
        std::vector<float> fine(tf.size(), 1e30f);
        for (int round = 0; round < 2; ++round)
            for (size_t q = 0; q < tf.size(); ++q) fine[q] = std::min(fine[q], time_fused(tf[q].second, 8));
        for (size_t q = 0; q < tf.size(); ++q)
            if (fine[q] < best_f) {
                best_f = fine[q];
                bf = tf[q].second;
            }
        best_f *= reps;   // back to the passes' unit: ms per reps launches
    } else {
        cudaGetLastError();
        c->err.clear();
    }
    const bool fused = best_f < best_h + best_e;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        const char* o = backup;
        for (auto& p : parts) {
            cudaMemcpyAsync(p.ptr, o, p.bytes, cudaMemcpyDeviceToDevice, c->stream);
            o += p.bytes;
        }
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(backup);
    MB_CUDA(c, cudaGetLastError());
    c->tune_h = bh;
    c->tune_e = be;
    c->tune_f = bf;
    c->use_fused = fused;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[{c->nx, c->ny, c->nz, c->p.npml}] = TuneSet{bh, be, bf, fused};
    }
    drop_graphs(c);
    return MB_OK;
}

int mb_get_single_pass(mb_ctx* c, int tune[4]) {
    if (int rc = check_ctx(c)) return rc;
    if (!tune) return fail(c, MB_ERR_ARG, "null output");
    tune[0] = c->use_fused ? 1 : 0;
    tune[1] = c->tune_f.block.x;
    tune[2] = c->tune_f.block.y;
    tune[3] = c->tune_f.kz;
    return MB_OK;
}

int mb_set_single_pass(mb_ctx* c, const int tune[4]) {
    if (int rc = check_ctx(c)) return rc;
    if (!tune) return fail(c, MB_ERR_ARG, "null input");
    if (tune[0] != 0 && tune[0] != 1) return fail(c, MB_ERR_ARG, "tune[0] must be 0 or 1");
    if (tune[0] == 0) {
        c->use_fused = false;
        drop_graphs(c);
        return MB_OK;
    }
    if (!mb::fused_tile_supported(tune[1], tune[2]) || tune[3] < 1)
        return fail(c, MB_ERR_ARG, "single-pass tiles are 32x4, 32x8, 64x4 or 64x8, kz >= 1");
    if (!mb::tma_e_supported(c->args))
        return fail(c, MB_ERR_ARG, "the single-pass step needs n_x % 16 == 0");
    if (int rc = ensure_second_copy(c)) return rc;
    const mb::PassTune t{mb::kVariantTma, dim3(tune[1], tune[2], 1), tune[3]};
    if (!fused_maps_for(c, t)) return fail(c, MB_ERR_ARG, "tensor maps of the single-pass step cannot be encoded");
    c->tune_f = t;
    c->use_fused = true;
    drop_graphs(c);
    return MB_OK;
}

int mb_get_tuning(mb_ctx* c, int tune_h[4], int tune_e[4]) {
    if (int rc = check_ctx(c)) return rc;
    if (!tune_h || !tune_e) return fail(c, MB_ERR_ARG, "null output");
    const mb::PassTune* src[2] = {&c->tune_h, &c->tune_e};
    int* dst[2] = {tune_h, tune_e};
    for (int q = 0; q < 2; ++q) {
        dst[q][0] = src[q]->variant;
        dst[q][1] = src[q]->block.x;
        dst[q][2] = src[q]->block.y;
        dst[q][3] = src[q]->variant == mb::kVariant3D ? (int)src[q]->block.z : src[q]->kz;
    }
    return MB_OK;
}

int mb_set_tuning(mb_ctx* c, const int tune_h[4], const int tune_e[4]) {
    if (int rc = check_ctx(c)) return rc;
    if (!tune_h || !tune_e) return fail(c, MB_ERR_ARG, "null input");
    mb::PassTune t[2];
    const int* src[2] = {tune_h, tune_e};
    for (int q = 0; q < 2; ++q) {
        const int* b = src[q];
        const bool tma = b[0] == mb::kVariantTma;
        const bool vec = b[0] == mb::kVariantVec;
        if (vec && !mb::vec_supported(c->args))
            return fail(c, MB_ERR_ARG, "the quad-vectorised passes need n_x % 4 == 0");
        if ((b[0] != mb::kVariant3D && b[0] != mb::kVariantZmarch && !vec && !tma) ||
            b[1] < 32 || b[1] % 32 || b[2] < 1 || b[3] < 1)
            return fail(c, MB_ERR_ARG,
                        "bad tuning: variant 0..3, x a multiple of 32, y, z >= 1");
        const int threads = b[1] * b[2] * (b[0] == mb::kVariant3D ? b[3] : 1);
        if (threads > (vec ? 256 : 512))
            return fail(c, MB_ERR_ARG, "at most 512 threads per block (256 for the quad variant)");
        t[q].variant = b[0];
        t[q].block = dim3(b[1], b[2], b[0] == mb::kVariant3D ? b[3] : 1);
        t[q].kz = b[0] == mb::kVariant3D ? 1 : b[3];
        if (tma && !tma_for(c, t[q]))
            return fail(c, MB_ERR_ARG, "the TMA passes need n_x % 16 == 0 and a tile of 32x4, 32x8, "
                                       "64x4, 64x8, 128x2 or 128x4");
    }
    c->tune_h = t[0];
    c->tune_e = t[1];
    drop_graphs(c);
    return MB_OK;
}

int mb_launch_stats(mb_ctx* c, int* per_step, int64_t* total) {
    if (int rc = check_ctx(c)) return rc;
    if (per_step) *per_step = launches_per_step(c, c->use_fused);
    if (total) *total = c->launches;
    return MB_OK;
}

}  // extern "C"
