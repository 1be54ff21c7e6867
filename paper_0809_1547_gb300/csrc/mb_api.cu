// C ABI of the Maxwell–Bloch FDTD library: context set-up, coefficient
// tables (FP64 on the host, FP32 on the device), materials, probes and
// sources, read-outs, state save / restore.  Stepping, the two field copies
// of the single-pass step and the autotuner are in mb_step.cu.
#include "mb_ctx.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>

using mb::kC0;
using mb::kEps0;
using mb::kHbar;
using mb::kPi;
using mb::kQe;

namespace mbi {

thread_local std::string g_err;
// allocations left before an injected failure (-1: none)
std::atomic<int> g_fail_alloc_after{-1};

bool inject_alloc_failure() {
    int v = g_fail_alloc_after.load();
    while (v >= 0) {
        if (g_fail_alloc_after.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

int fail(mb_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    g_err = msg;
    return code;
}


// Solve the 4x4 system A x = b (Gaussian elimination with partial pivoting).
void solve4(const double Ain[4][4], const double bin[4], double x[4]) {
    double A[4][5];
    for (int r = 0; r < 4; ++r) {
        for (int c = 0; c < 4; ++c) A[r][c] = Ain[r][c];
        A[r][4] = bin[r];
    }
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 5; ++c) std::swap(A[col][c], A[piv][c]);
        for (int r = col + 1; r < 4; ++r) {
            const double f = A[r][col] / A[col][col];
            for (int c = col; c < 5; ++c) A[r][c] -= f * A[col][c];
        }
    }
    for (int r = 3; r >= 0; --r) {
        double s = A[r][4];
        for (int c = r + 1; c < 4; ++c) s -= A[r][c] * x[c];
        x[r] = s / A[r][r];
    }
}

// CPML (Roden & Gedney 2000, kappa = 1) at positions x = i + half, i < n.
void cpml_table(int n, double half, int L, double dx, double dt, const mb_params& p,
                float* b, float* c) {
    const double eta0 = 1.0 / (kEps0 * kC0);
    const double sigma_max = p.pml_sigma_factor * (p.pml_order + 1.0) / (eta0 * dx);
    const double alpha_max = 2.0 * kPi * kEps0 * p.pml_alpha_rel * kC0 / p.lambda0;
    for (int i = 0; i < n; ++i) {
        b[i] = 0.0f;
        c[i] = 0.0f;
        if (L <= 0) continue;
        const double x = i + half;
        double depth = std::max((L - x) / L, (x - (n - L)) / (double)L);
        depth = std::min(1.0, std::max(0.0, depth));
        if (depth <= 0.0) continue;
        const double sigma = sigma_max * std::pow(depth, p.pml_order);
        const double alpha = alpha_max * (1.0 - depth);
        const double bb = std::exp(-(sigma + alpha) * dt / kEps0);
        b[i] = (float)bb;
        c[i] = (float)(sigma / (sigma + alpha) * (bb - 1.0));
    }
}

std::pair<int, int> interior(int n, int L) {
    return (n - 2 * L > 0) ? std::make_pair(L, n - L) : std::make_pair(0, n);
}

// E, H block (6 arrays) and CPML memories of copy p (0: the context's own
// arrays, 1: the single-pass step's second copy).
float* eh_of(const mb_ctx* c, int p) { return p ? c->d_fields2 : c->d_fields; }
float* psi_of(const mb_ctx* c, int p, int w) { return p ? c->d_psi2[w] : c->d_psi[w]; }

float* field_ptr(mb_ctx* c, int which) {
    // layout: ex ey ez hx hy hz (current copy), px py pz jx jy jz n1 n2 n3
    if (which < MB_EX || which > MB_N3 || which == MB_N0) return nullptr;
    const int slot = which < MB_N0 ? which : which - 1;
    if (slot < 6) return eh_of(c, c->parity) + (int64_t)slot * c->ncell;
    return c->d_fields + (int64_t)slot * c->ncell;
}

// Points the step arguments' E, H and CPML memories at copy p.
void point_args_at(mb::StepArgs& a, const mb_ctx* c, int p) {
    const int64_t N = c->ncell;
    float* F = eh_of(c, p);
    a.f.ex = F + 0 * N; a.f.ey = F + 1 * N; a.f.ez = F + 2 * N;
    a.f.hx = F + 3 * N; a.f.hy = F + 4 * N; a.f.hz = F + 5 * N;
    a.pml.psx = psi_of(c, p, 0);
    a.pml.psy = psi_of(c, p, 1);
    a.pml.psz = psi_of(c, p, 2);
}

double field_scale(const mb_ctx* c, int which) {
    if (which <= MB_EZ) return c->E0;
    if (which <= MB_HZ) return c->E0 / c->eta0;
    if (which <= MB_PZ) return kEps0 * c->E0;
    if (which <= MB_JZ) return kEps0 * c->E0 / c->dt;
    return c->N_a;
}

// The z-CPML region of the context's planes: the whole grid's CPML planes
// (k < L or k >= gnz - L in the grid's numbering) in local planes, and the
// layers the context stores for them (see DevCpml).
void z_cpml_bounds(const mb_ctx* c, mb::DevCpml& m) {
    const int L = c->p.npml;
    m.zlo = L - c->kz0;
    m.zhi = c->gnz - L - c->kz0;
    m.zs = std::max(0, m.zlo);
    m.zn = L ? m.zs + std::max(0, c->nz - m.zhi) : 0;
}

void build_args(mb_ctx* c) {
    mb::StepArgs& a = c->args;
    a.g = {c->nx, c->ny, c->nz, (uint32_t)c->nx * (uint32_t)c->ny, (uint32_t)c->ncell};
    float* F = c->d_fields;
    const int64_t N = c->ncell;
    a.f.px = F + 6 * N; a.f.py = F + 7 * N; a.f.pz = F + 8 * N;
    a.f.jx = F + 9 * N; a.f.jy = F + 10 * N; a.f.jz = F + 11 * N;
    a.f.n1 = F + 12 * N; a.f.n2 = F + 13 * N; a.f.n3 = F + 14 * N;
    a.f.mat = c->d_mat;
    a.f.inv_eps = c->dense_eps ? c->d_inv_eps : nullptr;
    a.f.lut_inv_eps = c->d_lut;
    a.f.n_lut = c->n_lut;
    a.f.ie0 = c->h_lut_ie[0];
    a.f.ie1 = c->h_lut_ie[1];
    const int L = c->p.npml;
    a.pml.L = L;
    z_cpml_bounds(c, a.pml);
    point_args_at(a, c, c->parity);
    const float* t = c->d_coef;
    const int n3[3] = {c->nx, c->ny, c->nz};
    const float** tabs[3][4] = {{&a.pml.bex, &a.pml.cex, &a.pml.bhx, &a.pml.chx},
                                {&a.pml.bey, &a.pml.cey, &a.pml.bhy, &a.pml.chy},
                                {&a.pml.bez, &a.pml.cez, &a.pml.bhz, &a.pml.chz}};
    for (int w = 0; w < 3; ++w)
        for (int q = 0; q < 4; ++q) {
            *tabs[w][q] = t;
            t += n3[w];
        }
    a.src = c->src;
    a.flux.on = 1;
    for (int w = 0; w < 3; ++w) {
        auto r = interior(n3[w], L);
        a.flux.r0[w] = r.first;
        a.flux.r1[w] = r.second;
        a.flux.plo[w] = r.first;
        a.flux.phi[w] = r.second;
    }
    if (c->slab) {
        // the whole grid's box in local planes, cut to the slab's own planes
        // (face planes outside them become -1: never met)
        const auto r = interior(c->gnz, L);
        const int lo = r.first - c->kz0, hi = r.second - c->kz0;
        a.flux.r0[2] = std::max(lo, c->own_lo);
        a.flux.r1[2] = std::min(hi, c->own_hi);
        a.flux.plo[2] = (lo >= c->own_lo && lo < c->own_hi) ? lo : -1;
        a.flux.phi[2] = (hi >= c->own_lo && hi < c->own_hi) ? hi : -1;
    }
    a.flux.acc = c->d_flux;
    a.S = (float)c->S;
    a.step_ctr = c->d_ctr;
    a.err = c->d_err;
    a.glist.cell = c->d_glist;
    a.glist.count = c->glist_count;
}

// Crank–Nicolson propagator of dN/dt = A N + e s, N = (N0, N1, N2, N3):
// M = L^-1 R, m = L^-1 e (times dt on use), L = I - (dt/2) A, R = I + (dt/2) A.
void cn_propagator(const mb_params& p, double W_p, double dt, double M[4][4], double m[4],
                   double Lm[4][4]) {
    double A[4][4] = {{0}};
    A[0][0] = -W_p;
    A[0][1] = 1.0 / p.tau10;
    A[1][1] = -1.0 / p.tau10;
    A[1][2] = 1.0 / p.tau21;
    A[2][2] = -1.0 / p.tau21;
    A[2][3] = 1.0 / p.tau32;
    A[3][3] = -1.0 / p.tau32;
    A[3][0] = W_p;
    double Rm[4][4];
    for (int r = 0; r < 4; ++r)
        for (int q = 0; q < 4; ++q) {
            Lm[r][q] = (r == q ? 1.0 : 0.0) - 0.5 * dt * A[r][q];
            Rm[r][q] = (r == q ? 1.0 : 0.0) + 0.5 * dt * A[r][q];
        }
    for (int q = 0; q < 4; ++q) {
        double col[4] = {Rm[0][q], Rm[1][q], Rm[2][q], Rm[3][q]}, x[4];
        solve4(Lm, col, x);
        for (int r = 0; r < 4; ++r) M[r][q] = x[r];
    }
    const double e[4] = {0.0, -1.0, 1.0, 0.0};
    solve4(Lm, e, m);
}

// The gain medium's step coefficients in device units (the fields of
// DevGain but the noise keys) for N_a atoms per m^3 pumped at W_p.
void gain_table(const mb_params& p, double dt, double dx, double N_a, double W_p, double E0,
                mb::DevGain& G) {
    const double w0 = 2.0 * kPi * kC0 / p.lambda0;
    const double dw = 2.0 * kPi * kC0 * p.dlambda / (p.lambda0 * p.lambda0);
    const double xi = 6.0 * kPi * kEps0 * kC0 * kC0 * kC0 / (w0 * w0 * p.tau21);
    const double a_se = p.a_se >= 0 ? p.a_se : w0 * (kQe * p.dipole_len) * std::sqrt(2.0 * dw);
    const double a = 0.5 * dw * dt;
    G.on = 1;
    G.cJ1 = (float)((1.0 - a) / (1.0 + a));
    G.cJE = (float)(dt * dt * xi * N_a / (kEps0 * (1.0 + a)));
    G.cJP = (float)((w0 * dt) * (w0 * dt) / (1.0 + a));
    G.cJN = (float)(dt * dt * a_se * std::sqrt(N_a / (dx * dx * dx * dt)) /
                    (kEps0 * E0 * (1.0 + a)));
    G.nfloor = (float)p.n_floor_rel;
    double M[4][4], m[4], Lm[4][4];
    cn_propagator(p, W_p, dt, M, m, Lm);
    const double smk = kEps0 * E0 * E0 / (kHbar * w0 * N_a);   // m s / N_a per S_pop
    for (int r = 0; r < 3; ++r) {
        G.g[r] = (float)M[r + 1][0];
        for (int q = 0; q < 3; ++q)
            G.G[r][q] = (float)(M[r + 1][q + 1] - M[r + 1][0] - (r == q ? 1.0 : 0.0));
        G.mk[r] = (float)(m[r + 1] * smk);
    }
}

void gain_coefficients(mb_ctx* c) {
    mb::DevGain& G = c->args.gain;
    std::memset(&G, 0, sizeof(G));
    if (c->N_a > 0.0) gain_table(c->p, c->dt, c->dx, c->N_a, c->W_p, c->E0, G);
    G.key0 = (uint32_t)(c->seed & 0xffffffffu);
    G.key1 = (uint32_t)(c->seed >> 32);
    G.cell0 = (uint32_t)((int64_t)c->kz0 * c->nx * c->ny);
}

int check_ctx_nojoin(mb_ctx* c) {
    if (!c) {
        g_err = "null context";
        return MB_ERR_ARG;
    }
    return MB_OK;
}

int check_ctx(mb_ctx* c) {
    if (int rc = check_ctx_nojoin(c)) return rc;
    mb::join_probes(c);
    return MB_OK;
}

std::vector<StatePart> state_parts(mb_ctx* c) {
    std::vector<StatePart> v;
    v.push_back({eh_of(c, c->parity), sizeof(float) * 6 * (size_t)c->ncell});
    v.push_back({c->d_fields + 6 * c->ncell, sizeof(float) * 9 * (size_t)c->ncell});
    for (int w = 0; w < 3; ++w)
        if (c->psi_elems[w]) v.push_back({psi_of(c, c->parity, w), sizeof(float) * c->psi_elems[w]});
    v.push_back({c->d_ctr, sizeof(long long) * 2});
    v.push_back({c->d_flux, sizeof(double) * 6 * mb::kFluxSlots});
    if (!c->probes.empty())
        v.push_back({c->d_probe_acc, sizeof(double2) * 3 * c->probes.size() * c->probe_nfreq});
    if (c->face.on && c->face_points) {
        v.push_back({c->d_face_acc, sizeof(double2) * 4 * (size_t)c->face_points * c->face.nfreq});
        v.push_back({c->d_face_acc32, sizeof(float2) * 4 * (size_t)c->face_points * c->face.nfreq});
    }
    for (const mb::DevPlaneProbe& q : c->planes)
        v.push_back({q.acc, sizeof(double2) * 3 * (size_t)q.nfreq * c->nx * c->ny});
    return v;
}

// Tensor maps for a TMA tuning over the current copy (encoded once per tile
// shape and copy), else nullptr.
const mb::TmaMaps* tma_for(mb_ctx* c, const mb::PassTune& t) {
    if (t.variant != mb::kVariantTma) return nullptr;
    const auto key = std::make_tuple((int)t.block.x, (int)t.block.y, c->parity);
    auto it = c->tma_maps.find(key);
    if (it != c->tma_maps.end()) return &it->second;
    mb::TmaMaps m;
    if (!mb::encode_tma(c->args, t.block.x, t.block.y, &m)) return nullptr;
    return &(c->tma_maps[key] = m);
}

// Device error flag (a bounded wait gave up): MB_ERR_TIMEOUT, flag cleared.
int check_device_error(mb_ctx* c) {
    int e = 0;
    MB_CUDA(c, cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (e) {
        cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
        return fail(c, MB_ERR_TIMEOUT, "a bounded device wait gave up (results of that step are invalid)");
    }
    return MB_OK;
}

// The probes of one step, after its E pass: point DFTs, face DFTs, plane DFTs
// of the fields in a (the context's arrays, or the single-pass step's second
// copy after the first step of a pair).
// ctr: the counter holding the step index of the fields sampled (the main
// counter, or the sample slot of a single-pass step's output copy).
void launch_probes(mb_ctx* c, const mb::StepArgs& a, const long long* ctr, cudaStream_t s) {
    mb::DevPointProbes pp{(int)c->probes.size(), c->probe_nfreq, c->d_probe_cell,
                          c->d_probe_omega, c->d_probe_acc};
    mb::launch_point_dft(pp, a.f, ctr, c->dt, s);
    mb::launch_face_dft(c->face, a.f, a.g, ctr, c->dt, s);
    for (const mb::DevPlaneProbe& q : c->planes) mb::launch_plane_dft(q, a.f, a.g, ctr, c->dt, s);
}

void launch_probes(mb_ctx* c) { launch_probes(c, c->args, c->d_ctr, c->stream); }

bool has_probes(const mb_ctx* c) { return !c->probes.empty() || c->face.on || !c->planes.empty(); }

void sum_flux_slots(const double* slots, double fl[6]) {
    for (int q = 0; q < 6; ++q) {
        double v = 0.0;
        for (int t = 0; t < mb::kFluxSlots; ++t) v += slots[q * mb::kFluxSlots + t];
        fl[q] = v;
    }
}

// Launches of one step: the field launches (2 for the two passes, 1 for the
// single-pass step) plus the probes.
int launches_per_step(const mb_ctx* c, bool fused) {
    return (fused ? 1 : 2) + (c->probes.empty() ? 0 : 1) + (c->face.on ? 1 : 0) + (int)c->planes.size();
}

void drop_graphs(mb_ctx* c) {
    for (int p = 0; p < 2; ++p) {
        if (c->graph_chunk[p]) cudaGraphExecDestroy(c->graph_chunk[p]);
        if (c->graph_one[p]) cudaGraphExecDestroy(c->graph_one[p]);
        c->graph_chunk[p] = c->graph_one[p] = nullptr;
    }
}

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, TuneSet> g_tune_cache;

}  // namespace mbi

using namespace mbi;

// (internal) message for mb_last_error(NULL) from calls without a context
void mb::set_thread_error(const std::string& msg) { g_err = msg; }

void mb::gain_pump_derivative(const mb_ctx* c, float dg[3], float dG[3][3], float dmk[3]) {
    // dM/dW = (dt/2) L^-1 A_W (I + M), dm/dW = (dt/2) L^-1 A_W m with
    // A_W = dA/dW_p (pump N0 -> N3), mapped to the reduced (n1, n2, n3) form
    // as the propagator itself.
    const double dt = c->dt;
    double M[4][4], m[4], Lm[4][4];
    cn_propagator(c->p, c->W_p, dt, M, m, Lm);
    double dM[4][4], dm[4];
    for (int q = 0; q < 4; ++q) {
        const double top = (q == 0 ? 1.0 : 0.0) + M[0][q];   // row 0 of (I + M)
        const double rhs[4] = {-0.5 * dt * top, 0.0, 0.0, 0.5 * dt * top};
        double x[4];
        solve4(Lm, rhs, x);
        for (int r = 0; r < 4; ++r) dM[r][q] = x[r];
    }
    {
        const double rhs[4] = {-0.5 * dt * m[0], 0.0, 0.0, 0.5 * dt * m[0]};
        solve4(Lm, rhs, dm);
    }
    const double w0 = 2.0 * kPi * kC0 / c->p.lambda0;
    const double smk = c->N_a > 0 ? kEps0 * c->E0 * c->E0 / (kHbar * w0 * c->N_a) : 0.0;
    for (int r = 0; r < 3; ++r) {
        dg[r] = (float)dM[r + 1][0];
        for (int q = 0; q < 3; ++q) dG[r][q] = (float)(dM[r + 1][q + 1] - dM[r + 1][0]);
        dmk[r] = (float)(dm[r + 1] * smk);
    }
}

const mb::TmaMaps* mb::tma_maps(mb_ctx* c, const mb::PassTune& t) { return tma_for(c, t); }

size_t mb::state_device_bytes(mb_ctx* c) {
    size_t total = 0;
    for (auto& p : state_parts(c)) total += p.bytes;
    return total;
}

int mb::state_snapshot(mb_ctx* c, void* d_dst) {
    char* o = static_cast<char*>(d_dst);
    for (auto& p : state_parts(c)) {
        MB_CUDA(c, cudaMemcpyAsync(o, p.ptr, p.bytes, cudaMemcpyDeviceToDevice, c->stream));
        o += p.bytes;
    }
    return MB_OK;
}

int mb::state_restore(mb_ctx* c, const void* d_src) {
    const char* o = static_cast<const char*>(d_src);
    for (auto& p : state_parts(c)) {
        MB_CUDA(c, cudaMemcpyAsync(p.ptr, o, p.bytes, cudaMemcpyDeviceToDevice, c->stream));
        o += p.bytes;
    }
    return MB_OK;
}

namespace mbi {

// Host side of mb_set_material (no device work): the material byte of each
// of the N cells (bits 0..6: id of its eps_r value, bit 7: gain cell when
// gain_on) into mat, the gain cells' indices in increasing order into glist
// (grown to glist_cap entries as needed, not zeroed), the distinct values in
// id order into lut_eps (empty when dense: more than 128 values, every id 0),
// and their count into n_gain.  Returns MB_OK, MB_ERR_MATERIALS (a value not
// finite or below 1; mat is then partly written) or MB_ERR_OOM.
int map_materials(const float* eps_map, const uint8_t* gain_mask, int64_t N, bool gain_on,
                  int max_threads, uint8_t* mat, std::unique_ptr<uint32_t[]>& glist, size_t& glist_cap,
                  std::vector<float>& lut_eps, bool& dense, size_t& n_gain) {
    // Material ids by the bit pattern of eps_r: up to 128 distinct values
    // share a LUT, more switch to a dense 1/eps map.  One pool of host
    // threads over chunks of cells, two passes with a barrier between.
    // Pass A: each thread validates its cells, gives them ids in a table of
    // its own (a packing holds a few values in long runs: the last value is
    // checked first, then the short table), sets the gain bit and counts its
    // gain cells.  Thread 0 then merges the tables in chunk order (ids =
    // order of first appearance) and places the threads' gain-list segments.
    // Pass B: each thread maps its ids to the merged ones and writes its gain
    // cells, in increasing order, into its segment.
    const int nthr = (int)std::max<int64_t>(1, std::min<int64_t>(
        {(int64_t)std::max(1u, std::thread::hardware_concurrency()), (int64_t)std::max(1, max_threads),
         N / (1 << 18) + 1}));
    std::vector<std::pair<int64_t, int64_t>> chunk(nthr);
    for (int t = 0; t < nthr; ++t) chunk[t] = {N * t / nthr, N * (t + 1) / nthr};
    std::vector<std::vector<uint32_t>> seen(nthr);
    std::vector<char> bad(nthr, 0), over(nthr, 0);
    std::vector<int64_t> ngain(nthr, 0), goff(nthr + 1, 0);
    auto find_key = [](const std::vector<uint32_t>& keys, uint32_t bits) -> int {
        for (size_t t = 0; t < keys.size(); ++t)
            if (keys[t] == bits) return (int)t;
        return -1;
    };
    std::vector<uint32_t> keys;
    bool any_bad = false, no_mem = false;
    dense = false;
    std::mutex mu;
    std::condition_variable cv;
    int arrived = 0;
    bool merged = false;
    auto body = [&](int t) {
        {
            std::vector<uint32_t>& tk = seen[t];
            uint32_t last = 0;
            int last_id = -1;
            int64_t cnt = 0;
            const int64_t end = chunk[t].second;
            const unsigned gon = gain_on ? 1u : 0u;
            for (int64_t q0 = chunk[t].first; q0 < end && !bad[t];) {
                // Blocks of 64 cells whose values are all among the (at most
                // four) already seen go through a branch-free loop the
                // compiler vectorizes; a block with a new or invalid value
                // takes the per-cell loop below.
                if (q0 + 64 <= end && tk.size() <= 4) {
                    uint32_t k[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu};
                    for (size_t u = 0; u < tk.size(); ++u) k[u] = tk[u];
                    const float* __restrict__ ep = eps_map + q0;
                    const uint8_t* __restrict__ gp = gain_mask + q0;
                    uint8_t* __restrict__ mp = mat + q0;
                    unsigned all = 1, ok = 1, gc = 0;
                    for (int u = 0; u < 64; ++u) {
                        uint32_t b;
                        std::memcpy(&b, ep + u, 4);
                        // 1 <= eps_r <= FLT_MAX: sign clear, 0x3f800000 <= bits < 0x7f800000
                        ok &= (b - 0x3f800000u) < 0x40000000u;
                        const unsigned m1 = b == k[1], m2 = b == k[2], m3 = b == k[3];
                        all &= (b == k[0]) | m1 | m2 | m3;
                        const unsigned g = gon & (gp[u] != 0);
                        mp[u] = (uint8_t)((m1 + 2 * m2 + 3 * m3) | (g << 7));
                        gc += g;
                    }
                    if (ok && all) {
                        cnt += gc;
                        q0 += 64;
                        continue;
                    }
                }
                const int64_t qe = std::min<int64_t>(end, q0 + 64);
                for (int64_t q = q0; q < qe; ++q) {
                    const float v = eps_map[q];
                    if (!(v >= 1.0f) || !std::isfinite(v)) {
                        bad[t] = 1;
                        break;
                    }
                    uint32_t bits;
                    std::memcpy(&bits, &v, 4);
                    if (last_id < 0 || bits != last) {
                        last = bits;
                        last_id = find_key(tk, bits);
                        if (last_id < 0) {
                            if (tk.size() < 128) {
                                last_id = (int)tk.size();
                                tk.push_back(bits);
                            } else {
                                over[t] = 1;   // more than 128 values: dense map
                                last_id = 0;
                            }
                        }
                    }
                    const bool g = gain_on && gain_mask[q] != 0;
                    mat[q] = (uint8_t)last_id | (g ? 0x80 : 0x00);
                    cnt += g;
                }
                q0 = qe;
            }
            ngain[t] = cnt;
        }
        {
            std::unique_lock<std::mutex> lk(mu);
            if (++arrived == nthr) {
                // every thread finished pass A: merge (on the last to arrive)
                for (int r = 0; r < nthr; ++r) any_bad |= bad[r] != 0;
                for (int r = 0; r < nthr && !dense; ++r) {
                    dense = over[r] != 0;
                    for (uint32_t bits : seen[r])
                        if (!dense && find_key(keys, bits) < 0) {
                            if (keys.size() == 128) {
                                dense = true;
                                break;
                            }
                            keys.push_back(bits);
                        }
                }
                for (int r = 0; r < nthr; ++r) goff[r + 1] = goff[r] + ngain[r];
                const size_t need = (size_t)std::max<int64_t>(goff[nthr], 1);
                if (!any_bad && glist_cap < need) {
                    glist.reset(new (std::nothrow) uint32_t[need]);
                    glist_cap = glist ? need : 0;
                    no_mem = !glist;
                }
                merged = true;
                cv.notify_all();
            } else {
                cv.wait(lk, [&] { return merged; });
            }
        }
        if (any_bad || no_mem) return;
        uint8_t remap[128];
        bool identity = true;
        for (size_t q = 0; q < seen[t].size(); ++q) {
            remap[q] = dense ? 0 : (uint8_t)find_key(keys, seen[t][q]);
            identity &= remap[q] == (uint8_t)q;
        }
        if (!identity)
            for (int64_t q = chunk[t].first; q < chunk[t].second; ++q)
                mat[q] = (uint8_t)(remap[mat[q] & 0x7f] | (mat[q] & 0x80));
        // gain cells in order, without a branch per cell: every index is
        // written and the position advances on gain cells; the loop ends when
        // the thread's segment is full, so no write leaves it
        uint32_t* out = glist.get() + goff[t];
        uint32_t* const out_end = glist.get() + goff[t + 1];
        for (int64_t q = chunk[t].first; q < chunk[t].second && out < out_end; ++q) {
            *out = (uint32_t)q;
            out += mat[q] >> 7;
        }
    };
    {
        std::vector<std::thread> pool;
        for (int t = 1; t < nthr; ++t) pool.emplace_back(body, t);
        body(0);
        for (auto& th : pool) th.join();
    }
    if (any_bad) return MB_ERR_MATERIALS;
    if (no_mem) return MB_ERR_OOM;
    lut_eps.clear();
    for (uint32_t bits : keys) {
        float v;
        std::memcpy(&v, &bits, 4);
        lut_eps.push_back(v);
    }
    n_gain = (size_t)goff[nthr];
    return MB_OK;
}

}  // namespace mbi

extern "C" {

void mb_default_params(mb_params* p) {
    if (!p) return;
    p->lambda0 = 590e-9;
    p->dlambda = 230e-9;
    p->tau32 = 100e-15;
    p->tau21 = 1e-9;
    p->tau10 = 100e-15;
    p->a_se = -1.0;
    p->dipole_len = 0.1e-9;
    p->n_floor_rel = 1e-9;
    p->npml = 8;
    p->pml_order = 3.0;
    p->pml_sigma_factor = 0.8;
    p->pml_alpha_rel = 0.1;
    p->n_ref = 1e24;
}

const char* mb_last_error(const mb_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_err.c_str();
}

static int check_create_args(mb_ctx** out, const int grid[3], double dx, double dt,
                             const mb_params* p, mb_params& prm) {
    if (!out || !grid) return fail(nullptr, MB_ERR_ARG, "null argument");
    *out = nullptr;
    if (grid[0] < 1 || grid[1] < 1 || grid[2] < 1) return fail(nullptr, MB_ERR_ARG, "grid sizes must be >= 1");
    const int64_t ncell = (int64_t)grid[0] * grid[1] * grid[2];
    if (ncell >= (int64_t(1) << 32)) return fail(nullptr, MB_ERR_ARG, "more than 2^32 cells");
    if (!(dx > 0) || !(dt > 0)) return fail(nullptr, MB_ERR_ARG, "dx and dt must be > 0");
    if (dt > dx / (kC0 * std::sqrt(3.0))) return fail(nullptr, MB_ERR_COURANT, "dt above the 3D Courant limit dx/(c sqrt 3)");
    mb_default_params(&prm);
    if (p) prm = *p;
    if (prm.npml < 0 || !(prm.lambda0 > 0) || !(prm.dlambda > 0) || !(prm.tau21 > 0) ||
        !(prm.tau32 > 0) || !(prm.tau10 > 0) || !(prm.n_ref > 0) || prm.n_floor_rel < 0)
        return fail(nullptr, MB_ERR_ARG, "invalid parameter");
    return MB_OK;
}

// A context over grid (local planes); its z-window is planes kz0 .. kz0 +
// grid[2] - 1 of a grid of gnz planes, of which [own_lo, own_hi) are its own
// (the whole grid: gnz = grid[2], kz0 = own_lo = 0, own_hi = grid[2]).
static int create_ctx(mb_ctx** out, const int grid[3], int gnz, int kz0, int own_lo, int own_hi,
                      bool slab, double dx, double dt, const mb_params& prm, void* cuda_stream) {
    const int64_t ncell = (int64_t)grid[0] * grid[1] * grid[2];
    mb_ctx* c = new mb_ctx();
    c->nx = grid[0];
    c->ny = grid[1];
    c->nz = grid[2];
    c->ncell = ncell;
    c->slab = slab;
    c->gnz = gnz;
    c->kz0 = kz0;
    c->own_lo = own_lo;
    c->own_hi = own_hi;
    c->dx = dx;
    c->dt = dt;
    c->p = prm;
    c->eta0 = 1.0 / (kEps0 * kC0);
    c->S = kC0 * dt / dx;
    const double w0 = 2.0 * kPi * kC0 / prm.lambda0;
    c->E0 = std::sqrt(kHbar * w0 * prm.n_ref / kEps0);
    auto bail = [&](int code) {
        mb_destroy(c);
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(fail(nullptr, MB_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e)));
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(fail(nullptr, MB_ERR_CUDA, cudaGetErrorString(e)));
        c->own_stream = true;
    }
    auto alloc = [&](void** ptr, size_t bytes) -> int {
        if (bytes == 0) { *ptr = nullptr; return MB_OK; }
        cudaError_t ae = inject_alloc_failure() ? cudaErrorMemoryAllocation : cudaMalloc(ptr, bytes);
        if (ae != cudaSuccess) {
            cudaGetLastError();
            return fail(nullptr, MB_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        }
        c->dev_bytes += bytes;
        return MB_OK;
    };
    int rc;
    if ((rc = alloc((void**)&c->d_fields, sizeof(float) * 15 * (size_t)ncell))) return bail(rc);
    if ((rc = alloc((void**)&c->d_mat, (size_t)ncell))) return bail(rc);
    if ((rc = alloc((void**)&c->d_lut, sizeof(float) * 256))) return bail(rc);
    const int L = prm.npml;
    c->psi_elems[0] = L ? (size_t)4 * c->nz * c->ny * 2 * L : 0;
    c->psi_elems[1] = L ? (size_t)4 * c->nz * 2 * L * c->nx : 0;
    mb::DevCpml zb{};
    z_cpml_bounds(c, zb);
    c->psi_elems[2] = (size_t)4 * zb.zn * c->ny * c->nx;
    for (int w = 0; w < 3; ++w)
        if ((rc = alloc((void**)&c->d_psi[w], sizeof(float) * c->psi_elems[w]))) return bail(rc);
    const size_t ncoef = 4 * (size_t)(c->nx + c->ny + c->nz);
    if ((rc = alloc((void**)&c->d_coef, sizeof(float) * ncoef))) return bail(rc);
    if ((rc = alloc((void**)&c->d_ctr, sizeof(long long) * 4))) return bail(rc);
    if ((rc = alloc((void**)&c->d_flux, sizeof(double) * 6 * mb::kFluxSlots))) return bail(rc);
    if ((rc = alloc((void**)&c->d_flux_out, sizeof(double) * 6))) return bail(rc);
    c->n_partial = 1024;
    if ((rc = alloc((void**)&c->d_partial, sizeof(double) * c->n_partial))) return bail(rc);
    if ((rc = alloc((void**)&c->d_energy, sizeof(double)))) return bail(rc);
    if ((rc = alloc((void**)&c->d_nonfinite, sizeof(int)))) return bail(rc);
    if ((rc = alloc((void**)&c->d_err, sizeof(int)))) return bail(rc);

    // CPML tables, zeroed state, eps_r = 1 (material 0), no gain.
    std::vector<float> coef(ncoef);
    float* t = coef.data();
    const int n3[3] = {c->nx, c->ny, c->nz};
    for (int w = 0; w < 2; ++w) {
        cpml_table(n3[w], 0.0, L, dx, dt, prm, t, t + n3[w]);
        cpml_table(n3[w], 0.5, L, dx, dt, prm, t + 2 * n3[w], t + 3 * n3[w]);
        t += 4 * n3[w];
    }
    {
        // z: the whole grid's profile, the context's planes of it
        std::vector<float> zt(4 * (size_t)gnz);
        cpml_table(gnz, 0.0, L, dx, dt, prm, zt.data(), zt.data() + gnz);
        cpml_table(gnz, 0.5, L, dx, dt, prm, zt.data() + 2 * gnz, zt.data() + 3 * gnz);
        for (int q = 0; q < 4; ++q)
            std::copy(zt.begin() + (size_t)q * gnz + kz0, zt.begin() + (size_t)q * gnz + kz0 + c->nz,
                      t + (size_t)q * c->nz);
    }
    std::vector<float> lut(256, 1.0f);
    c->h_lut_eps.assign(128, 1.0f);
#define MB_CREATE_CUDA(call)                                                               \
    do {                                                                                   \
        cudaError_t ce_ = (call);                                                          \
        if (ce_ != cudaSuccess) return bail(fail(nullptr, MB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(ce_))); \
    } while (0)
    MB_CREATE_CUDA(cudaMemcpy(c->d_coef, coef.data(), sizeof(float) * ncoef, cudaMemcpyHostToDevice));
    MB_CREATE_CUDA(cudaMemcpy(c->d_lut, lut.data(), sizeof(float) * 256, cudaMemcpyHostToDevice));
    MB_CREATE_CUDA(cudaMemset(c->d_fields, 0, sizeof(float) * 15 * (size_t)ncell));
    MB_CREATE_CUDA(cudaMemset(c->d_mat, 0, (size_t)ncell));
    for (int w = 0; w < 3; ++w)
        if (c->psi_elems[w]) MB_CREATE_CUDA(cudaMemset(c->d_psi[w], 0, sizeof(float) * c->psi_elems[w]));
    MB_CREATE_CUDA(cudaMemset(c->d_ctr, 0, sizeof(long long) * 4));
    MB_CREATE_CUDA(cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking));
    MB_CREATE_CUDA(cudaMemset(c->d_err, 0, sizeof(int)));
    MB_CREATE_CUDA(cudaMemset(c->d_flux, 0, sizeof(double) * 6 * mb::kFluxSlots));
#undef MB_CREATE_CUDA
    c->face.on = 0;
    build_args(c);
    gain_coefficients(c);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find({c->nx, c->ny, c->nz, L});
        if (it != g_tune_cache.end()) {
            c->tune_h = it->second.h;
            c->tune_e = it->second.e;
            c->tune_f = it->second.f;
            c->use_fused = it->second.fused;   // second copy allocated at the first step
        }
    }
    *out = c;
    return MB_OK;
}

int mb_create(mb_ctx** out, const int grid[3], double dx, double dt, const mb_params* p,
              void* cuda_stream) {
    mb_params prm;
    if (int rc = check_create_args(out, grid, dx, dt, p, prm)) return rc;
    return create_ctx(out, grid, grid[2], 0, 0, grid[2], false, dx, dt, prm, cuda_stream);
}

int mb_create_slab(mb_ctx** out, const int grid[3], int z_begin, int z_end, double dx, double dt,
                   const mb_params* p, void* cuda_stream) {
    mb_params prm;
    if (int rc = check_create_args(out, grid, dx, dt, p, prm)) return rc;
    const int gnz = grid[2], L = prm.npml;
    if (z_begin < 0 || z_end > gnz || z_begin >= z_end)
        return fail(nullptr, MB_ERR_ARG, "need 0 <= z_begin < z_end <= grid[2]");
    // a cut plane c leaves ghost planes c - 1 and c, which must lie outside
    // the z-CPML (their CPML memories along z are not exchanged)
    auto bad_cut = [&](int cut) { return cut < L + 1 || cut > gnz - L - 1; };
    if ((z_begin > 0 && bad_cut(z_begin)) || (z_end < gnz && bad_cut(z_end)))
        return fail(nullptr, MB_ERR_ARG, "cut planes must lie in [npml + 1, grid[2] - npml - 1]");
    const int below = z_begin > 0 ? 1 : 0, above = z_end < gnz ? 1 : 0;
    const int local[3] = {grid[0], grid[1], z_end - z_begin + below + above};
    return create_ctx(out, local, gnz, z_begin - below, below, below + z_end - z_begin,
                      true, dx, dt, prm, cuda_stream);
}

int mb_slab_info(mb_ctx* c, int info[4]) {
    if (int rc = check_ctx_nojoin(c)) return rc;
    if (!info) return fail(c, MB_ERR_ARG, "null output");
    info[0] = c->gnz;
    info[1] = c->kz0;
    info[2] = c->own_lo;
    info[3] = c->own_hi;
    return MB_OK;
}

int mb_destroy(mb_ctx* c) {
    if (!c) return MB_OK;
    if (c->stream) {
        mb::join_probes(c);
        cudaStreamSynchronize(c->stream);
    }
    drop_graphs(c);
    void* bufs[] = {c->d_fields, c->d_mat, c->d_inv_eps, c->d_lut, c->d_psi[0], c->d_psi[1],
                    c->d_psi[2], c->d_coef, c->d_ctr, c->d_flux, c->d_partial, c->d_energy,
                    c->d_nonfinite, c->d_probe_cell, c->d_probe_omega, c->d_probe_acc,
                    c->d_face_omega, c->d_face_acc, c->d_face_acc32, c->d_glist, c->d_glist_scratch,
                    c->d_upload, c->d_keys, c->d_src_wave, c->d_err,
                    c->d_fields2, c->d_psi2[0], c->d_psi2[1], c->d_psi2[2], c->d_flux_out};
    for (void* b : bufs)
        if (b) cudaFree(b);
    for (const mb::DevPlaneProbe& q : c->planes) {
        cudaFree(const_cast<double*>(q.omega));
        cudaFree(q.acc);
    }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    if (c->aux_stream) cudaStreamDestroy(c->aux_stream);
    for (cudaEvent_t ev : c->fork_ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : c->join_ev) cudaEventDestroy(ev);
    for (int q = 0; q < 2; ++q) {
        if (c->probe_fork[q]) cudaEventDestroy(c->probe_fork[q]);
        if (c->probe_done[q]) cudaEventDestroy(c->probe_done[q]);
    }
    delete c;
    return MB_OK;
}

int mb_set_material(mb_ctx* c, const float* eps_map, const uint8_t* gain_mask, double N_a,
                    double pump) {
    if (int rc = check_ctx(c)) return rc;
    NvtxRange range("mb_set_material");
    if (!eps_map || !gain_mask) return fail(c, MB_ERR_ARG, "null eps_map or gain_mask");
    if (!(N_a >= 0) || !(pump >= 0) || !std::isfinite(N_a) || !std::isfinite(pump))
        return fail(c, MB_ERR_ARG, "N_a and pump must be finite and >= 0");
    const int64_t N = c->ncell;
    // The map on the device: the eps_r map and the gain mask uploaded into
    // scratch, their distinct values found (checked before any state of the
    // context changes), the table sorted on the host, the material bytes and
    // the gain-cell list built from it.
    auto grow = [&](void** p, size_t& have, size_t need) -> bool {
        if (have >= need && *p) return true;
        if (*p) cudaFree(*p);
        *p = nullptr;
        have = 0;
        if (cudaMalloc(p, need) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        have = need;
        return true;
    };
    const size_t up_bytes = 5 * (size_t)N;
    const size_t key_bytes = 2 * sizeof(uint32_t) * mb::kMatKeys + 2 * sizeof(int);
    if (!grow((void**)&c->d_upload, c->upload_bytes, up_bytes) ||
        !grow((void**)&c->d_keys, c->keys_bytes, key_bytes))
        return fail(c, MB_ERR_OOM, "material map scratch allocation failed");
    float* d_eps = reinterpret_cast<float*>(c->d_upload);
    uint8_t* d_gain = c->d_upload + 4 * (size_t)N;
    uint32_t* d_first = c->d_keys + mb::kMatKeys;
    int* d_flags = reinterpret_cast<int*>(c->d_keys + 2 * mb::kMatKeys);
    MB_CUDA(c, cudaMemsetAsync(c->d_keys, 0xff, 2 * sizeof(uint32_t) * mb::kMatKeys, c->stream));
    MB_CUDA(c, cudaMemsetAsync(d_flags, 0, 2 * sizeof(int), c->stream));
    MB_CUDA(c, cudaMemcpyAsync(d_eps, eps_map, sizeof(float) * (size_t)N, cudaMemcpyHostToDevice, c->stream));
    MB_CUDA(c, cudaMemcpyAsync(d_gain, gain_mask, (size_t)N, cudaMemcpyHostToDevice, c->stream));
    mb::launch_mat_keys(d_eps, N, c->d_keys, d_first, d_flags, c->stream);
    uint32_t h_keys[2 * mb::kMatKeys + 2];
    MB_CUDA(c, cudaMemcpyAsync(h_keys, c->d_keys, key_bytes, cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    const int* h_flags = reinterpret_cast<const int*>(h_keys + 2 * mb::kMatKeys);
    if (h_flags[0]) return fail(c, MB_ERR_MATERIALS, "eps_r must be finite and >= 1");
    const bool dense = h_flags[1] != 0;
    // the table in order of first appearance in the map (the ids do not
    // depend on the order in which the device filled it, and equal those of
    // the host statement of the map, mb_material_map)
    std::vector<float> lut_eps;
    std::vector<uint32_t> keys;
    if (!dense) {
        std::vector<std::pair<uint32_t, uint32_t>> kf;   // (first cell, bits)
        for (int q = 0; q < mb::kMatKeys && h_keys[q] != mb::kNoKey; ++q)
            kf.push_back({h_keys[mb::kMatKeys + q], h_keys[q]});
        std::sort(kf.begin(), kf.end());
        for (const auto& p : kf) keys.push_back(p.second);
        for (uint32_t k : keys) {
            float v;
            std::memcpy(&v, &k, 4);
            lut_eps.push_back(v);
        }
        if (!keys.empty())
            MB_CUDA(c, cudaMemcpyAsync(c->d_keys, keys.data(), sizeof(uint32_t) * keys.size(),
                                       cudaMemcpyHostToDevice, c->stream));
    }
    std::vector<float> lut(256, 1.0f);
    c->h_lut_eps.assign(128, 1.0f);
    for (size_t q = 0; q < lut_eps.size(); ++q) {
        lut[q] = (float)(1.0 / (double)lut_eps[q]);
        lut[128 + q] = lut_eps[q];
        c->h_lut_eps[q] = lut_eps[q];
    }
    if (dense && !c->d_inv_eps) {
        cudaError_t e = cudaMalloc((void**)&c->d_inv_eps, sizeof(float) * (size_t)N);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(c, MB_ERR_OOM, "dense eps map allocation failed"); }
        c->dev_bytes += sizeof(float) * (size_t)N;
    }
    const size_t nsc = mb::gain_list_scratch(N);
    if (nsc > c->glist_scratch_n) {
        if (c->d_glist_scratch) cudaFree(c->d_glist_scratch);
        c->d_glist_scratch = nullptr;
        c->glist_scratch_n = 0;
        cudaError_t e = cudaMalloc((void**)&c->d_glist_scratch, sizeof(uint32_t) * nsc);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(c, MB_ERR_OOM, "gain list allocation failed"); }
        c->glist_scratch_n = nsc;
    }
    mb::launch_mat_ids(d_eps, d_gain, N, c->d_keys, (int)keys.size(), dense, N_a > 0.0, c->d_mat,
                       c->d_inv_eps, c->stream);
    MB_CUDA(c, cudaMemcpyAsync(c->d_lut, lut.data(), sizeof(float) * 256, cudaMemcpyHostToDevice, c->stream));
    // gain cells in increasing order: the two-pass step's Lorentz blocks run over this list
    mb::launch_gain_count(c->d_mat, N, c->d_glist_scratch, c->stream);
    uint32_t n_gain32 = 0;
    MB_CUDA(c, cudaMemcpyAsync(&n_gain32, c->d_glist_scratch + (nsc - 2), sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    const size_t n_gain = n_gain32;
    if (n_gain > c->glist_capacity || !c->d_glist) {
        if (c->d_glist) {
            cudaFree(c->d_glist);
            c->dev_bytes -= sizeof(uint32_t) * c->glist_capacity;
            c->d_glist = nullptr;
        }
        const size_t cap = n_gain ? n_gain : 1;
        cudaError_t e = cudaMalloc((void**)&c->d_glist, sizeof(uint32_t) * cap);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(c, MB_ERR_OOM, "gain list allocation failed"); }
        c->glist_capacity = cap;
        c->dev_bytes += sizeof(uint32_t) * cap;
    }
    if (n_gain) mb::launch_gain_scatter(c->d_mat, N, c->d_glist_scratch, c->d_glist, c->stream);
    // dense maps (no table) take the per-cell array; n_lut counts the table
    c->n_lut = dense ? 128 : (int)lut_eps.size();
    c->h_lut_ie[0] = lut[0];
    c->h_lut_ie[1] = lut[1];
    c->dense_eps = dense;
    c->N_a = N_a;
    c->W_p = pump;
    c->glist_count = (uint32_t)n_gain;
    // reset P, J and the populations (N0 = N_a, n1 = n2 = n3 = 0)
    MB_CUDA(c, cudaMemsetAsync(c->d_fields + 6 * N, 0, sizeof(float) * 9 * (size_t)N, c->stream));
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    c->have_material = true;
    build_args(c);
    gain_coefficients(c);
    drop_graphs(c);
    return MB_OK;
}

int mb_set_seed(mb_ctx* c, uint64_t seed) {
    if (int rc = check_ctx(c)) return rc;
    c->seed = seed;
    c->args.gain.key0 = (uint32_t)(seed & 0xffffffffu);
    c->args.gain.key1 = (uint32_t)(seed >> 32);
    drop_graphs(c);
    return MB_OK;
}

int mb_add_point_probe(mb_ctx* c, const int ijk[3], int n_freq, double lam_min, double lam_max,
                       int* probe_id) {
    if (int rc = check_ctx(c)) return rc;
    if (!ijk || n_freq < 1 || !(lam_min > 0) || !(lam_max > 0))
        return fail(c, MB_ERR_ARG, "bad point-probe arguments");
    if (ijk[0] < 0 || ijk[0] >= c->nx || ijk[1] < 0 || ijk[1] >= c->ny || ijk[2] < 0 || ijk[2] >= c->nz)
        return fail(c, MB_ERR_ARG, "probe cell outside the grid");
    if (!c->probes.empty() && n_freq != c->probe_nfreq)
        return fail(c, MB_ERR_ARG, "all point probes of a context share one bin count");
    cudaStreamSynchronize(c->stream);
    mb::PointProbeHost pr;
    pr.cell = ijk[0] + (int64_t)c->nx * (ijk[1] + (int64_t)c->ny * ijk[2]);
    pr.nfreq = n_freq;
    for (int k = 0; k < n_freq; ++k) {
        const double lam = n_freq == 1 ? lam_min : lam_min + (lam_max - lam_min) * k / (n_freq - 1);
        pr.lam.push_back(lam);
        pr.omega.push_back(2.0 * kPi * kC0 / lam);
    }
    const size_t P = c->probes.size() + 1;
    int64_t* d_cell = nullptr;
    double* d_om = nullptr;
    double2* d_acc = nullptr;
    MB_CUDA(c, cudaMalloc((void**)&d_cell, sizeof(int64_t) * P));
    MB_CUDA(c, cudaMalloc((void**)&d_om, sizeof(double) * P * n_freq));
    MB_CUDA(c, cudaMalloc((void**)&d_acc, sizeof(double2) * 3 * P * n_freq));
    MB_CUDA(c, cudaMemset(d_acc, 0, sizeof(double2) * 3 * P * n_freq));
    if (P > 1) {
        MB_CUDA(c, cudaMemcpy(d_acc, c->d_probe_acc, sizeof(double2) * 3 * (P - 1) * n_freq, cudaMemcpyDeviceToDevice));
    }
    c->probes.push_back(pr);
    std::vector<int64_t> cells;
    std::vector<double> om;
    for (auto& q : c->probes) {
        cells.push_back(q.cell);
        om.insert(om.end(), q.omega.begin(), q.omega.end());
    }
    MB_CUDA(c, cudaMemcpy(d_cell, cells.data(), sizeof(int64_t) * P, cudaMemcpyHostToDevice));
    MB_CUDA(c, cudaMemcpy(d_om, om.data(), sizeof(double) * P * n_freq, cudaMemcpyHostToDevice));
    if (c->d_probe_cell) cudaFree(c->d_probe_cell);
    if (c->d_probe_omega) cudaFree(c->d_probe_omega);
    if (c->d_probe_acc) cudaFree(c->d_probe_acc);
    c->d_probe_cell = d_cell;
    c->d_probe_omega = d_om;
    c->d_probe_acc = d_acc;
    c->probe_nfreq = n_freq;
    if (probe_id) *probe_id = (int)(P - 1);
    drop_graphs(c);
    return MB_OK;
}

int mb_add_face_probes(mb_ctx* c, int stride, int every, int n_freq, double lam_min, double lam_max) {
    if (int rc = check_ctx(c)) return rc;
    if (stride < 1 || every < 1 || n_freq < 1 || n_freq > 4096 || !(lam_min > 0) || !(lam_max > 0))
        return fail(c, MB_ERR_ARG, "bad face-probe arguments (1 <= n_freq <= 4096)");
    cudaStreamSynchronize(c->stream);
    if (c->d_face_acc) { cudaFree(c->d_face_acc); c->d_face_acc = nullptr; }
    if (c->d_face_acc32) { cudaFree(c->d_face_acc32); c->d_face_acc32 = nullptr; }
    if (c->d_face_omega) { cudaFree(c->d_face_omega); c->d_face_omega = nullptr; }
    mb::DevFaceProbes& F = c->face;
    std::memset(&F, 0, sizeof(F));
    const int n3[3] = {c->nx, c->ny, c->nz};
    const int L = c->p.npml;
    int64_t off = 0;
    for (int face = 0; face < 6; ++face) {
        const int ax = face / 2;
        auto r = interior(n3[ax], L);
        F.plane[face] = (face % 2) ? r.second : r.first;
        // transverse axes (a, b): x-face (y, z), y-face (x, z) by point order, z-face (x, y)
        const int ta = ax == 0 ? 1 : 0;
        const int tb = ax == 2 ? 1 : 2;
        auto ra = interior(n3[ta], L), rb = interior(n3[tb], L);
        int na = (ra.second - ra.first + stride - 1) / stride;
        int nb = (rb.second - rb.first + stride - 1) / stride;
        F.r0a[face] = ra.first;
        F.r0b[face] = rb.first;
        if (c->slab) {
            // the whole grid's lattice of points, cut to the slab's own planes
            // (local coordinates): x and y faces keep the lattice rows whose
            // z lies in them (their samples stay in the plane), a z face
            // belongs to the slab owning the plane below it, where its H is
            // sampled (the plane itself, holding E, is then own too, or the
            // grid's end: a cut never falls next to the z-CPML)
            const int zlo = c->kz0 + c->own_lo, zhi = c->kz0 + c->own_hi;   // whole-grid planes
            if (ax == 2) {
                auto rz = interior(c->gnz, L);
                const int gp = (face % 2) ? rz.second : rz.first;
                const int gq = std::max(gp - 1, 0);
                F.plane[face] = gp - c->kz0;
                if (gq < zlo || gq >= zhi) nb = 0;
            } else {
                auto rz = interior(c->gnz, L);
                const int nbg = (rz.second - rz.first + stride - 1) / stride;
                const int qlo = std::max(0, (zlo - rz.first + stride - 1) / stride);
                const int qhi = std::min(nbg, std::max(0, (zhi - rz.first + stride - 1) / stride));
                nb = std::max(0, qhi - qlo);
                F.r0b[face] = rz.first + qlo * stride - c->kz0;
            }
        }
        F.na[face] = na;
        F.npts[face] = na * nb;
        F.offset[face] = (int)off;
        off += (int64_t)na * nb;
    }
    F.on = 1;
    F.stride = stride;
    F.every = every;
    F.nfreq = n_freq;
    F.pts_per_block = 32;
    c->face_points = off;
    c->face_lam.clear();
    std::vector<double> om;
    for (int k = 0; k < n_freq; ++k) {
        const double lam = n_freq == 1 ? lam_min : lam_min + (lam_max - lam_min) * k / (n_freq - 1);
        c->face_lam.push_back(lam);
        om.push_back(2.0 * kPi * kC0 / lam);
    }
    MB_CUDA(c, cudaMalloc((void**)&c->d_face_omega, sizeof(double) * n_freq));
    MB_CUDA(c, cudaMemcpy(c->d_face_omega, om.data(), sizeof(double) * n_freq, cudaMemcpyHostToDevice));
    const size_t accn = 4 * (size_t)off * n_freq;
    MB_CUDA(c, cudaMalloc((void**)&c->d_face_acc, sizeof(double2) * (accn ? accn : 1)));
    MB_CUDA(c, cudaMemset(c->d_face_acc, 0, sizeof(double2) * (accn ? accn : 1)));
    MB_CUDA(c, cudaMalloc((void**)&c->d_face_acc32, sizeof(float2) * (accn ? accn : 1)));
    MB_CUDA(c, cudaMemset(c->d_face_acc32, 0, sizeof(float2) * (accn ? accn : 1)));
    F.omega = c->d_face_omega;
    F.acc = c->d_face_acc;
    F.acc32 = c->d_face_acc32;
    drop_graphs(c);
    return MB_OK;
}

int mb_set_source(mb_ctx* c, const int ijk[3], int comp, double lam, double t0, double tau, double amp) {
    if (int rc = check_ctx(c)) return rc;
    if (amp == 0.0) {
        c->src.on = 0;
        c->args.src = c->src;
        drop_graphs(c);
        return MB_OK;
    }
    if (!ijk || comp < 0 || comp > 2 || !(lam > 0) || !(tau > 0) || !std::isfinite(amp))
        return fail(c, MB_ERR_ARG, "bad source arguments");
    if (ijk[0] < 0 || ijk[0] >= c->nx || ijk[1] < 0 || ijk[1] >= c->ny || ijk[2] < 0 || ijk[2] >= c->nz)
        return fail(c, MB_ERR_ARG, "source cell outside the grid");
    // Tabulate the scaled current J dt/(eps0 E0) at t = (n + 1/2) dt in FP64
    // over the steps where |t - t0| < 12 tau (the envelope is below 1e-62 outside).
    const double amp_s = amp * c->dt / (kEps0 * c->E0);
    const double ws = 2.0 * kPi * kC0 / lam;
    const long long n0 = std::max(0LL, (long long)std::floor((t0 - 12.0 * tau) / c->dt - 0.5));
    const long long n1 = (long long)std::ceil((t0 + 12.0 * tau) / c->dt - 0.5) + 1;
    if (n1 <= n0 || n1 - n0 > (1LL << 24)) return fail(c, MB_ERR_ARG, "source window empty or too long");
    std::vector<float> wave((size_t)(n1 - n0));
    for (long long n = n0; n < n1; ++n) {
        const double t = ((double)n + 0.5) * c->dt - t0;
        const double e = t / tau;
        wave[(size_t)(n - n0)] = (float)(amp_s * std::sin(ws * t) * std::exp(-e * e));
    }
    cudaStreamSynchronize(c->stream);
    if (c->d_src_wave) {
        cudaFree(c->d_src_wave);
        c->d_src_wave = nullptr;
    }
    MB_CUDA(c, cudaMalloc((void**)&c->d_src_wave, sizeof(float) * wave.size()));
    MB_CUDA(c, cudaMemcpy(c->d_src_wave, wave.data(), sizeof(float) * wave.size(), cudaMemcpyHostToDevice));
    c->src.on = 1;
    c->src.comp = comp;
    c->src.cell = ijk[0] + (int64_t)c->nx * (ijk[1] + (int64_t)c->ny * ijk[2]);
    c->src.n0 = n0;
    c->src.count = (int)(n1 - n0);
    c->src.wave = c->d_src_wave;
    c->args.src = c->src;
    drop_graphs(c);
    return MB_OK;
}

int mb_set_source_cw(mb_ctx* c, const int ijk[3], int comp, double lam, double t0, double tau,
                     double amp, int n_steps) {
    if (int rc = check_ctx(c)) return rc;
    if (amp == 0.0) return mb_set_source(c, ijk, comp, lam, t0, tau, 0.0);
    if (!ijk || comp < 0 || comp > 2 || !(lam > 0) || !(tau > 0) || !std::isfinite(amp) ||
        !(t0 >= 0) || n_steps < 1 || n_steps > (1 << 24))
        return fail(c, MB_ERR_ARG, "bad CW source arguments");
    if (ijk[0] < 0 || ijk[0] >= c->nx || ijk[1] < 0 || ijk[1] >= c->ny || ijk[2] < 0 || ijk[2] >= c->nz)
        return fail(c, MB_ERR_ARG, "source cell outside the grid");
    // n_steps steps from the first one whose t_{n+1/2} >= t0, tabulated in FP64
    const double amp_s = amp * c->dt / (kEps0 * c->E0);
    const double ws = 2.0 * kPi * kC0 / lam;
    const long long n0 = std::max(0LL, (long long)std::ceil(t0 / c->dt - 0.5));
    std::vector<float> wave((size_t)n_steps);
    for (long long q = 0; q < n_steps; ++q) {
        const double t = ((double)(n0 + q) + 0.5) * c->dt - t0;
        const double e = t / tau;
        wave[(size_t)q] = t < 0 ? 0.0f : (float)(amp_s * std::sin(ws * t) * (1.0 - std::exp(-e * e)));
    }
    cudaStreamSynchronize(c->stream);
    if (c->d_src_wave) {
        cudaFree(c->d_src_wave);
        c->d_src_wave = nullptr;
    }
    MB_CUDA(c, cudaMalloc((void**)&c->d_src_wave, sizeof(float) * wave.size()));
    MB_CUDA(c, cudaMemcpy(c->d_src_wave, wave.data(), sizeof(float) * wave.size(), cudaMemcpyHostToDevice));
    c->src.on = 1;
    c->src.comp = comp;
    c->src.cell = ijk[0] + (int64_t)c->nx * (ijk[1] + (int64_t)c->ny * ijk[2]);
    c->src.n0 = n0;
    c->src.count = n_steps;
    c->src.wave = c->d_src_wave;
    c->args.src = c->src;
    drop_graphs(c);
    return MB_OK;
}

int mb_add_plane_probe(mb_ctx* c, int k, int every, int n_freq, double lam_min, double lam_max,
                       int* probe_id) {
    if (int rc = check_ctx(c)) return rc;
    if (k < 0 || k >= c->nz || every < 1 || n_freq < 1 || n_freq > mb::kPlaneMaxFreq ||
        !(lam_min > 0) || !(lam_max > 0) || !probe_id)
        return fail(c, MB_ERR_ARG, "bad plane-probe arguments (1 <= n_freq <= 64, 0 <= k < n_z)");
    std::vector<double> lam, om;
    for (int q = 0; q < n_freq; ++q) {
        const double l = n_freq == 1 ? lam_min : lam_min + (lam_max - lam_min) * q / (n_freq - 1);
        lam.push_back(l);
        om.push_back(2.0 * kPi * kC0 / l);
    }
    cudaStreamSynchronize(c->stream);
    double* d_om = nullptr;
    double2* d_acc = nullptr;
    const size_t accn = 3 * (size_t)n_freq * c->nx * c->ny;
    cudaError_t e = cudaMalloc((void**)&d_om, sizeof(double) * n_freq);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_acc, sizeof(double2) * accn);
    if (e == cudaSuccess) e = cudaMemcpy(d_om, om.data(), sizeof(double) * n_freq, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_acc, 0, sizeof(double2) * accn);
    if (e != cudaSuccess) {
        if (d_om) cudaFree(d_om);
        if (d_acc) cudaFree(d_acc);
        return fail(c, e == cudaErrorMemoryAllocation ? MB_ERR_OOM : MB_ERR_CUDA, cudaGetErrorString(e));
    }
    c->planes.push_back(mb::DevPlaneProbe{k, every, n_freq, d_om, d_acc});
    c->plane_lam.push_back(lam);
    *probe_id = (int)c->planes.size() - 1;
    drop_graphs(c);
    return MB_OK;
}

int mb_plane_mode_map(mb_ctx* c, int probe_id, int bin, double* out_map) {
    if (int rc = check_ctx(c)) return rc;
    if (probe_id < 0 || probe_id >= (int)c->planes.size() || !out_map)
        return fail(c, MB_ERR_ARG, "bad plane probe");
    const mb::DevPlaneProbe& q = c->planes[probe_id];
    if (bin < 0 || bin >= q.nfreq) return fail(c, MB_ERR_ARG, "bad frequency bin");
    const size_t nxy = (size_t)c->nx * c->ny;
    std::vector<double2> acc(3 * nxy);
    MB_CUDA(c, cudaMemcpyAsync(acc.data(), q.acc + (size_t)bin * 3 * nxy, sizeof(double2) * 3 * nxy,
                               cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    const double w = c->E0 * q.every * c->dt;   // scaled sample -> V/m, times the DFT weight
    for (size_t p = 0; p < nxy; ++p) {
        double v = 0.0;
        for (int comp = 0; comp < 3; ++comp) {
            const double2 a = acc[comp * nxy + p];
            v += a.x * a.x + a.y * a.y;
        }
        out_map[p] = v * w * w;
    }
    return check_device_error(c);
}

int mb_plane_energy_density(mb_ctx* c, int k, double* out) {
    if (int rc = check_ctx(c)) return rc;
    if (k < 0 || k >= c->nz || !out) return fail(c, MB_ERR_ARG, "bad plane");
    const size_t nxy = (size_t)c->nx * c->ny;
    double* d = nullptr;
    MB_CUDA(c, cudaMalloc((void**)&d, sizeof(double) * nxy));
    mb::launch_plane_energy(c->args.f, c->args.g, k, c->d_lut + 128, d, c->stream);
    cudaError_t e = cudaMemcpyAsync(out, d, sizeof(double) * nxy, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return fail(c, MB_ERR_CUDA, cudaGetErrorString(e));
    const double u0 = kEps0 * c->E0 * c->E0;
    for (size_t p = 0; p < nxy; ++p) out[p] *= u0;
    return check_device_error(c);
}

// The six face energies (J) summed and scaled on the device into d_flux_out.
void enqueue_flux_out(mb_ctx* c) {
    const double f = c->dt * c->E0 * (c->E0 / c->eta0) * c->dx * c->dx;
    mb::launch_flux_sum(c->d_flux, c->d_flux_out, f, c->stream);
}

int mb_flux(mb_ctx* c, double* out_flux6) {
    if (int rc = check_ctx(c)) return rc;
    if (!out_flux6) return fail(c, MB_ERR_ARG, "null output");
    enqueue_flux_out(c);
    MB_CUDA(c, cudaMemcpyAsync(out_flux6, c->d_flux_out, sizeof(double) * 6, cudaMemcpyDeviceToHost,
                               c->stream));
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int mb_flux_async(mb_ctx* c, double* host_out6) {
    // the face sums are written by the field steps on the context's stream
    // only, so this read need not wait for probes on the second stream
    if (int rc = check_ctx_nojoin(c)) return rc;
    if (!host_out6) return fail(c, MB_ERR_ARG, "null output");
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host_out6) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer) {
        // page-locked host memory: the summing kernel writes it directly
        const double f = c->dt * c->E0 * (c->E0 / c->eta0) * c->dx * c->dx;
        mb::launch_flux_sum(c->d_flux, static_cast<double*>(at.devicePointer), f, c->stream);
        MB_CUDA(c, cudaGetLastError());
        return MB_OK;
    }
    cudaGetLastError();   // a failed attribute query leaves an error behind
    enqueue_flux_out(c);
    MB_CUDA(c, cudaMemcpyAsync(host_out6, c->d_flux_out, sizeof(double) * 6, cudaMemcpyDeviceToHost,
                               c->stream));
    return MB_OK;
}

int mb_join_probes(mb_ctx* c) { return check_ctx(c); }

int mb_reset_probes(mb_ctx* c) {
    if (int rc = check_ctx(c)) return rc;   // after the probe launches still running
    if (!c->probes.empty())
        MB_CUDA(c, cudaMemsetAsync(c->d_probe_acc, 0, sizeof(double2) * 3 * c->probes.size() * c->probe_nfreq,
                                   c->stream));
    if (c->face.on && c->face_points) {
        const size_t accn = 4 * (size_t)c->face_points * c->face.nfreq;
        MB_CUDA(c, cudaMemsetAsync(c->d_face_acc, 0, sizeof(double2) * accn, c->stream));
        MB_CUDA(c, cudaMemsetAsync(c->d_face_acc32, 0, sizeof(float2) * accn, c->stream));
    }
    for (const mb::DevPlaneProbe& q : c->planes)
        MB_CUDA(c, cudaMemsetAsync(q.acc, 0, sizeof(double2) * 3 * (size_t)q.nfreq * c->nx * c->ny, c->stream));
    return MB_OK;
}

int mb_synchronize(mb_ctx* c) {
    if (int rc = check_ctx(c)) return rc;
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    return check_device_error(c);
}

int mb_get_step(mb_ctx* c, int64_t* n) {
    if (int rc = check_ctx(c)) return rc;
    if (!n) return fail(c, MB_ERR_ARG, "null output");
    *n = c->n;
    return MB_OK;
}

int mb_probe_spectrum(mb_ctx* c, int probe_id, double* out_S, double* out_lam) {
    if (int rc = check_ctx(c)) return rc;
    if (probe_id < 0 || probe_id >= (int)c->probes.size() || !out_S)
        return fail(c, MB_ERR_ARG, "bad probe id or null output");
    const int K = c->probe_nfreq;
    std::vector<double2> acc(3 * (size_t)K);
    MB_CUDA(c, cudaMemcpyAsync(acc.data(), c->d_probe_acc + (size_t)probe_id * 3 * K,
                               sizeof(double2) * 3 * K, cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    const double f = c->E0 * c->dt;
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int q = 0; q < 3; ++q) {
            const double2 v = acc[(size_t)q * K + k];
            s += (v.x * v.x + v.y * v.y) * f * f;
        }
        out_S[k] = s;
        if (out_lam) out_lam[k] = c->probes[probe_id].lam[k];
    }
    return MB_OK;
}

int mb_face_spectrum(mb_ctx* c, int face, double* out_S, double* out_lam) {
    if (int rc = check_ctx(c)) return rc;
    if (!c->face.on) return fail(c, MB_ERR_STATE, "no face probes");
    if (face < 0 || face > 5 || !out_S) return fail(c, MB_ERR_ARG, "bad face or null output");
    const int K = c->face.nfreq;
    const int np = c->face.npts[face];
    std::vector<double2> acc((size_t)np * 4 * K);
    std::vector<float2> acc32((size_t)np * 4 * K);
    if (np) {
        const size_t at = (size_t)c->face.offset[face] * 4 * K;
        MB_CUDA(c, cudaMemcpyAsync(acc.data(), c->d_face_acc + at, sizeof(double2) * acc.size(),
                                   cudaMemcpyDeviceToHost, c->stream));
        MB_CUDA(c, cudaMemcpyAsync(acc32.data(), c->d_face_acc32 + at, sizeof(float2) * acc32.size(),
                                   cudaMemcpyDeviceToHost, c->stream));
        MB_CUDA(c, cudaStreamSynchronize(c->stream));
        // the FP64 sums plus the FP32 sums since their last flush
        for (size_t q = 0; q < acc.size(); ++q) {
            acc[q].x += (double)acc32[q].x;
            acc[q].y += (double)acc32[q].y;
        }
    }
    const double w = c->face.every * c->dt;
    const double scale = (c->E0 * w) * (c->E0 / c->eta0 * w) * std::pow(c->face.stride * c->dx, 2);
    const double sign = (face % 2) ? 1.0 : -1.0;
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int q = 0; q < np; ++q) {
            const double2 Ea = acc[((size_t)q * 4 + 0) * K + k], Eb = acc[((size_t)q * 4 + 1) * K + k];
            const double2 Ha = acc[((size_t)q * 4 + 2) * K + k], Hb = acc[((size_t)q * 4 + 3) * K + k];
            // Re(Ea conj(Hb) - Eb conj(Ha))
            s += (Ea.x * Hb.x + Ea.y * Hb.y) - (Eb.x * Ha.x + Eb.y * Ha.y);
        }
        out_S[k] = sign * s * scale;
        if (out_lam) out_lam[k] = c->face_lam[k];
    }
    return MB_OK;
}

int mb_energy(mb_ctx* c, double* out_U, double* out_flux6) {
    if (int rc = check_ctx(c)) return rc;
    if (!out_U) return fail(c, MB_ERR_ARG, "null output");
    MB_CUDA(c, cudaMemsetAsync(c->d_nonfinite, 0, sizeof(int), c->stream));
    // the context's own planes (all of them but a z-slab's ghost planes)
    const int64_t off = (int64_t)c->own_lo * c->nx * c->ny;
    const int64_t own = (int64_t)(c->own_hi - c->own_lo) * c->nx * c->ny;
    mb::DevFields f = c->args.f;
    for (float** q : {&f.ex, &f.ey, &f.ez, &f.hx, &f.hy, &f.hz, &f.px, &f.py, &f.pz, &f.jx, &f.jy,
                      &f.jz, &f.n1, &f.n2, &f.n3})
        *q += off;
    f.mat += off;
    if (f.inv_eps) f.inv_eps += off;
    mb::launch_energy(f, own, c->d_lut + 128, c->d_partial, c->n_partial, c->d_nonfinite,
                      c->d_energy, c->stream);
    MB_CUDA(c, cudaGetLastError());
    double U = 0, slots[6 * mb::kFluxSlots], fl[6];
    int bad = 0;
    MB_CUDA(c, cudaMemcpyAsync(&U, c->d_energy, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(c, cudaMemcpyAsync(slots, c->d_flux, sizeof(slots), cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(c, cudaMemcpyAsync(&bad, c->d_nonfinite, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    sum_flux_slots(slots, fl);
    *out_U = 0.5 * kEps0 * c->E0 * c->E0 * c->dx * c->dx * c->dx * U;
    if (out_flux6) {
        const double f = c->dt * c->E0 * (c->E0 / c->eta0) * c->dx * c->dx;
        for (int q = 0; q < 6; ++q) out_flux6[q] = fl[q] * f;
    }
    if (bad) return fail(c, MB_ERR_NONFINITE, "non-finite field values");
    return check_device_error(c);
}

int mb_gain_list(mb_ctx* c, uint32_t* host_out, int64_t* count) {
    if (int rc = check_ctx(c)) return rc;
    if (!count) return fail(c, MB_ERR_ARG, "null count");
    if (!c->have_material) return fail(c, MB_ERR_STATE, "no material set");
    *count = (int64_t)c->glist_count;
    if (!host_out || c->glist_count == 0) return MB_OK;
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    MB_CUDA(c, cudaMemcpy(host_out, c->d_glist, sizeof(uint32_t) * c->glist_count, cudaMemcpyDeviceToHost));
    return MB_OK;
}

int mb_get_material(mb_ctx* c, uint8_t* host_out) {
    if (int rc = check_ctx(c)) return rc;
    if (!host_out) return fail(c, MB_ERR_ARG, "null output");
    if (!c->have_material) return fail(c, MB_ERR_STATE, "no material set");
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    MB_CUDA(c, cudaMemcpy(host_out, c->d_mat, (size_t)c->ncell, cudaMemcpyDeviceToHost));
    return MB_OK;
}

int mb_get_cpml(mb_ctx* c, int axis, double* host_out, size_t* count) {
    if (int rc = check_ctx(c)) return rc;
    if (axis < 0 || axis > 2) return fail(c, MB_ERR_ARG, "axis must be 0, 1 or 2");
    const size_t n = c->psi_elems[axis];
    if (count) *count = n;
    if (!host_out || n == 0) return MB_OK;
    std::vector<float> tmp(n);
    MB_CUDA(c, cudaMemcpyAsync(tmp.data(), psi_of(c, c->parity, axis), sizeof(float) * n,
                               cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    // planes f = 0, 1 hold E-update memories (H differences), f = 2, 3 the
    // H-update ones (E differences): psi_E = psi_E,s E0 / (eta0 dx),
    // psi_H = psi_H,s E0 / dx
    const size_t per_f = n / 4;
    const double se = c->E0 / (c->eta0 * c->dx), sh = c->E0 / c->dx;
    for (size_t q = 0; q < n; ++q) host_out[q] = (q / per_f < 2 ? se : sh) * (double)tmp[q];
    return MB_OK;
}

int mb_get_field(mb_ctx* c, int which, float* host_out) {
    if (int rc = check_ctx(c)) return rc;
    if (!host_out || which < 0 || which >= MB_NUM_FIELDS) return fail(c, MB_ERR_ARG, "bad field id or null output");
    const int64_t N = c->ncell;
    std::vector<float> tmp((size_t)N);
    if (which == MB_N0) {
        std::vector<float> a((size_t)N), b((size_t)N), d((size_t)N);
        std::vector<uint8_t> m((size_t)N, 0);
        MB_CUDA(c, cudaMemcpyAsync(a.data(), field_ptr(c, MB_N1), 4 * N, cudaMemcpyDeviceToHost, c->stream));
        MB_CUDA(c, cudaMemcpyAsync(b.data(), field_ptr(c, MB_N2), 4 * N, cudaMemcpyDeviceToHost, c->stream));
        MB_CUDA(c, cudaMemcpyAsync(d.data(), field_ptr(c, MB_N3), 4 * N, cudaMemcpyDeviceToHost, c->stream));
        if (c->have_material)
            MB_CUDA(c, cudaMemcpyAsync(m.data(), c->d_mat, (size_t)N, cudaMemcpyDeviceToHost, c->stream));
        MB_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int64_t q = 0; q < N; ++q)
            host_out[q] = (m[q] & 0x80) ? (float)(c->N_a * (1.0 - (double)a[q] - (double)b[q] - (double)d[q])) : 0.0f;
        return MB_OK;
    }
    MB_CUDA(c, cudaMemcpyAsync(tmp.data(), field_ptr(c, which), 4 * N, cudaMemcpyDeviceToHost, c->stream));
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    const double s = field_scale(c, which);
    for (int64_t q = 0; q < N; ++q) host_out[q] = (float)(s * (double)tmp[q]);
    return MB_OK;
}

int mb_set_field(mb_ctx* c, int which, const float* host_in) {
    if (int rc = check_ctx(c)) return rc;
    if (!host_in || which < 0 || which >= MB_NUM_FIELDS) return fail(c, MB_ERR_ARG, "bad field id or null input");
    if (which == MB_N0) return fail(c, MB_ERR_ARG, "N0 is derived and cannot be set");
    if (which >= MB_N1 && !(c->N_a > 0)) return fail(c, MB_ERR_STATE, "populations need N_a > 0");
    const int64_t N = c->ncell;
    const double s = 1.0 / field_scale(c, which);
    std::vector<float> tmp((size_t)N);
    for (int64_t q = 0; q < N; ++q) tmp[q] = (float)(s * (double)host_in[q]);
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    MB_CUDA(c, cudaMemcpy(field_ptr(c, which), tmp.data(), 4 * N, cudaMemcpyHostToDevice));
    return MB_OK;
}

int mb_get_field_device(mb_ctx* c, int which, float* dev_out, double* scale) {
    if (int rc = check_ctx(c)) return rc;
    if (!dev_out || which < 0 || which >= MB_NUM_FIELDS || which == MB_N0)
        return fail(c, MB_ERR_ARG, "bad field id (N0 is not stored) or null output");
    MB_CUDA(c, cudaMemcpyAsync(dev_out, field_ptr(c, which), 4 * c->ncell, cudaMemcpyDeviceToDevice, c->stream));
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    if (scale) *scale = field_scale(c, which);
    return MB_OK;
}

int mb_save_state(mb_ctx* c, void* host_blob, size_t* bytes) {
    if (int rc = check_ctx(c)) return rc;
    if (!bytes) return fail(c, MB_ERR_ARG, "null size");
    auto parts = state_parts(c);
    size_t total = 4 * sizeof(int64_t);
    for (auto& p : parts) total += p.bytes;
    if (!host_blob) {
        *bytes = total;
        return MB_OK;
    }
    if (*bytes < total) return fail(c, MB_ERR_ARG, "blob too small");
    char* o = (char*)host_blob;
    const int64_t hdr[4] = {0x4D42464454445331LL, c->ncell, (int64_t)parts.size(), c->n};
    std::memcpy(o, hdr, sizeof(hdr));
    o += sizeof(hdr);
    for (auto& p : parts) {
        MB_CUDA(c, cudaMemcpyAsync(o, p.ptr, p.bytes, cudaMemcpyDeviceToHost, c->stream));
        o += p.bytes;
    }
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    *bytes = total;
    return MB_OK;
}

int mb_load_state(mb_ctx* c, const void* host_blob, size_t bytes) {
    if (int rc = check_ctx(c)) return rc;
    if (!host_blob) return fail(c, MB_ERR_ARG, "null blob");
    auto parts = state_parts(c);
    size_t total = 4 * sizeof(int64_t);
    for (auto& p : parts) total += p.bytes;
    const int64_t* hdr = (const int64_t*)host_blob;
    if (bytes != total || hdr[0] != 0x4D42464454445331LL || hdr[1] != c->ncell || hdr[2] != (int64_t)parts.size())
        return fail(c, MB_ERR_ARG, "blob does not match this context's layout");
    const char* o = (const char*)host_blob + 4 * sizeof(int64_t);
    MB_CUDA(c, cudaStreamSynchronize(c->stream));
    for (auto& p : parts) {
        MB_CUDA(c, cudaMemcpy(p.ptr, o, p.bytes, cudaMemcpyHostToDevice));
        o += p.bytes;
    }
    c->n = hdr[3];
    return MB_OK;
}

void mb_debug_fail_alloc(int n) { g_fail_alloc_after.store(n < 0 ? -1 : n); }

int mb_device_bytes(mb_ctx* c, size_t* bytes) {
    if (int rc = check_ctx(c)) return rc;
    if (!bytes) return fail(c, MB_ERR_ARG, "null output");
    *bytes = c->dev_bytes;
    return MB_OK;
}

int mb_host_tables(const int grid[3], double dx, double dt, const mb_params* p, double N_a,
                   double pump, float* out_cpml, float* out_gain, double* out_E0) {
    if (!grid || grid[0] < 1 || grid[1] < 1 || grid[2] < 1 || !(dx > 0) || !(dt > 0) ||
        !(N_a >= 0) || !(pump >= 0) || !out_cpml || !out_gain || !out_E0) {
        g_err = "bad host-table arguments";
        return MB_ERR_ARG;
    }
    mb_params prm;
    if (p) prm = *p;
    else mb_default_params(&prm);
    float* t = out_cpml;
    for (int w = 0; w < 3; ++w) {
        cpml_table(grid[w], 0.0, prm.npml, dx, dt, prm, t, t + grid[w]);
        cpml_table(grid[w], 0.5, prm.npml, dx, dt, prm, t + 2 * grid[w], t + 3 * grid[w]);
        t += 4 * grid[w];
    }
    const double w0 = 2.0 * kPi * kC0 / prm.lambda0;
    const double E0 = std::sqrt(kHbar * w0 * prm.n_ref / kEps0);
    mb::DevGain G;
    std::memset(&G, 0, sizeof(G));
    if (N_a > 0.0) gain_table(prm, dt, dx, N_a, pump, E0, G);
    float* o = out_gain;
    *o++ = G.cJ1;
    *o++ = G.cJE;
    *o++ = G.cJP;
    *o++ = G.cJN;
    *o++ = G.nfloor;
    for (int r = 0; r < 3; ++r) *o++ = G.g[r];
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) *o++ = G.G[r][q];
    for (int r = 0; r < 3; ++r) *o++ = G.mk[r];
    *out_E0 = E0;
    return MB_OK;
}

int mb_material_map(const float* eps_map, const uint8_t* gain_mask, int64_t n, int gain_on,
                    int max_threads, uint8_t* out_mat, uint32_t* out_glist, int64_t* out_n_gain,
                    float* out_lut_eps, int* out_n_values, int* out_dense) {
    if (!eps_map || !gain_mask || n < 1 || !out_mat || !out_glist || !out_n_gain || !out_lut_eps ||
        !out_n_values || !out_dense) {
        g_err = "bad material-map arguments";
        return MB_ERR_ARG;
    }
    std::unique_ptr<uint32_t[]> glist;
    size_t cap = 0, n_gain = 0;
    std::vector<float> lut;
    bool dense = false;
    const int rc = map_materials(eps_map, gain_mask, n, gain_on != 0, max_threads, out_mat, glist, cap,
                                 lut, dense, n_gain);
    if (rc) {
        g_err = rc == MB_ERR_OOM ? "host gain-list buffer allocation failed" : "eps_r must be finite and >= 1";
        return rc;
    }
    if (n_gain) std::memcpy(out_glist, glist.get(), sizeof(uint32_t) * n_gain);
    *out_n_gain = (int64_t)n_gain;
    for (size_t q = 0; q < lut.size(); ++q) out_lut_eps[q] = lut[q];
    *out_n_values = (int)lut.size();
    *out_dense = dense ? 1 : 0;
    return MB_OK;
}

int mb_philox4x32_10(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, int n) {
    if (!ctr || !key || !out || n < 0) return fail(nullptr, MB_ERR_ARG, "bad philox arguments");
    if (n == 0) return MB_OK;
    uint4 *d_in = nullptr, *d_out = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_in, sizeof(uint4) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_out, sizeof(uint4) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemcpy(d_in, ctr, sizeof(uint4) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        mb::launch_philox(d_in, key[0], key[1], d_out, n, 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(uint4) * (size_t)n, cudaMemcpyDeviceToHost);
    if (d_in) cudaFree(d_in);
    if (d_out) cudaFree(d_out);
    if (e != cudaSuccess) return fail(nullptr, MB_ERR_CUDA, std::string("philox: ") + cudaGetErrorString(e));
    return MB_OK;
}

}  // extern "C"
