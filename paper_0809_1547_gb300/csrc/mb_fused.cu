// Single-pass Maxwell–Bloch step: the H half-step, the Lorentz / Langevin
// update of the gain cells and the E / population update of one time step in
// one launch, so each cell's E and H cross HBM once per step (read one copy,
// write the other) instead of twice.
//
// A block owns a BX x BY tile of (i, j) columns and walks planes k0 .. k1-1.
// One thread streams, S - 1 planes ahead, each plane's E (with a one-cell
// halo on every side), H^{n-1/2} (with its -x/-y halo) and material tile from
// the source copy into an S-slot shared-memory ring (cp.async.bulk.tensor on
// mbarriers).  Plane k then takes four steps:
//   1. H^{n+1/2} of the tile's own cells (E of planes k and k+1), written to
//      the destination copy and to a shared tile; threads of the first warps
//      also compute H^{n+1/2} of the row j = y0-1 and the column i = x0-1,
//      which the E update of the tile's edge cells needs (the neighbouring
//      tiles compute the same values from the same inputs, bit for bit);
//   2. for gain cells, J^{n+1/2} and P^{n+1} (E^n from the ring, P, J and the
//      populations prefetched one plane ahead with cp.async), in place;
//   3. after a block barrier, E^{n+1} from the shared H tile and the own H of
//      plane k-1 (registers), the populations N^{n+1}, and in blocks that
//      hold face cells of the flux box their outward Poynting terms (summed
//      per warp and plane into shared partials, added to the FP64 face slots
//      once per block);
//   4. a barrier frees the ring slot for plane k + S.
// The first plane of a block needs H^{n+1/2} of plane k0-1 at its own cells:
// recomputed from the source copy (never written: the block below owns it).
// Because no block writes what another reads, the launch needs no ordering
// between blocks.  Every cell update is the helpers of the two-pass launches,
// so the result equals theirs bit for bit.
#include "mb_host.h"
#include "mb_tiles.cuh"
#include "mb_tma.cuh"

#include <cudaTypedefs.h>

#include <algorithm>

namespace mb {

template <int BX, int BY>
struct FusedLayout {
    static constexpr int kEX = BX + 8, kEY = BY + 2;   // E box from (x0-4, y0-1)
    static constexpr int kHX = BX + 4, kHY = BY + 1;   // H box from (x0-4, y0-1)
    static constexpr int kEW = kEX * kEY, kHW = kHX * kHY, kMW = BX * BY;
    static constexpr int kEBytes = (kEW * 4 + 127) / 128 * 128;
    static constexpr int kHBytes = (kHW * 4 + 127) / 128 * 128;
    static constexpr int kMBytes = (kMW + 127) / 128 * 128;
    static constexpr int kStage = 3 * kEBytes + 3 * kHBytes + kMBytes;
    static constexpr int kTxE = 3 * kEW * 4;                  // top stage: E only
    static constexpr int kTx = kTxE + 3 * kHW * 4 + kMW;
    // H^{n+1/2} of the tile with its -x/-y halo: [3][BY+1][BX+1]
    static constexpr int kNX = BX + 1, kNW = (BX + 1) * (BY + 1);
    static constexpr int kNBytes = (3 * kNW * 4 + 127) / 128 * 128;
    // P, J, n1..n3 of gain cells, two planes (cp.async double buffer)
    static constexpr int kGBytes = 2 * 9 * kMW * 4;
    static constexpr int smem_bytes(int stages) {
        return stages * kStage + kGBytes + kNBytes + 64 + 128;
    }
};

// Planes [k0, k1) of z block q of a launch with nq z blocks, for chunks of
// kz planes (nzb = ceil(nz / kz) of them; the last one may be shorter).
// Issue order: chunk 0, chunk nzb-1 (the two that hold the z-CPML), chunks
// 1 .. nzb-3, then chunk nzb-2 as two halves (nq = nzb + 1 when nzb >= 3
// and kz >= 2, else nq = nzb and chunks in the first order).
__host__ __device__ inline int fused_z_blocks(int nz, int kz) {
    const int nzb = (nz + kz - 1) / kz;
    return (nzb >= 3 && kz >= 2) ? nzb + 1 : nzb;
}
__device__ __forceinline__ void fused_chunk(int q, int nq, int nz, int kz, int& k0, int& k1) {
    const int nzb = (nz + kz - 1) / kz;
    int c = q == 0 ? 0 : (q == 1 ? nzb - 1 : q - 1);
    int lo = 0, hi = kz;
    if (nq == nzb + 1 && q >= nzb - 1) {   // the two halves of chunk nzb - 2
        c = nzb - 2;
        const int h = kz / 2;
        lo = q == nzb - 1 ? 0 : h;
        hi = q == nzb - 1 ? h : kz;
    }
    k0 = c * kz + lo;
    k1 = min(nz, c * kz + hi);
}

template <int BX, int BY, int S>
__global__ void __launch_bounds__(BX * BY) k_step_fused(StepArgs a, DevPing d,
                                                        const __grid_constant__ TmaFusedMaps maps,
                                                        int kz) {
    using Lay = FusedLayout<BX, BY>;
    constexpr int T = BX * BY;
    static_assert(BX + BY <= T, "the halo row and column need BX + BY threads");
    constexpr int NW = T / 32;
    extern __shared__ unsigned char smem_raw[];
    __shared__ float wfl[6][NW];   // per-warp face-flux partials
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float* gbuf = reinterpret_cast<float*>(smem + S * Lay::kStage);
    float* hn = reinterpret_cast<float*>(smem + S * Lay::kStage + Lay::kGBytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S * Lay::kStage + Lay::kGBytes + Lay::kNBytes);
    static_assert(BX % 8 == 0 && BY % 4 == 0, "x-edge tiles map warps onto 8 x 4 cells");
    const int tid = threadIdx.x + BX * threadIdx.y;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    // The thread's cell (tx, ty) in the tile.  In tiles that hold x-CPML
    // columns a warp covers 8 columns x 4 rows, so that the slab's columns
    // fill whole warps and the other warps skip the slab's work as a body;
    // elsewhere a warp covers one row.  Each warp access still covers whole
    // 32-byte sectors; the cell updates are the same either way.
    const bool xedge = a.pml.L > 0 && (x0 < a.pml.L || x0 + BX > a.g.nx - a.pml.L);
    const int wq = tid >> 5, ln = tid & 31;
    const int tx = xedge ? 8 * (wq % (BX / 8)) + (ln & 7) : tid % BX;
    const int ty = xedge ? 4 * (wq / (BX / 8)) + (ln >> 3) : tid / BX;
    const int tcell = tx + BX * ty;   // the cell's place in the tile's row-major shared arrays
    const int i = x0 + tx, j = y0 + ty;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const uint32_t nxy = a.g.nxy;
    const bool valid = i < nx && j < ny;
    // The planes of the block (fused_chunk): the z-CPML chunks, the
    // heaviest, are issued first and the last-issued chunk is cut in two, so
    // the launch does not end on heavy or long blocks.
    int k0, k1;
    fused_chunk(blockIdx.z, gridDim.z, nz, kz, k0, k1);
    const int planes = k1 - k0, total = planes + 1;
    const long long n = a.step_ctr[0];
    const bool face = tile_on_face(a.flux, x0, x0 + BX, y0, y0 + BY, k0, k1);
    // the tile with its halo row and column touches an x or y CPML slab
    const bool pml_xy = tile_in_xy_slab(a, x0 - 1, BX + 1, y0 - 1, BY + 1);
    const bool gain_on = a.gain.on;
    const DevFields& f = a.f;

    // The E box's lines are read again by the neighbouring tiles (its halo
    // rows and columns) and by the block of the next z chunk (its top
    // plane): they are kept in L2 ahead of the rest (evict-last), and the
    // block's writes, which nothing in the launch reads again, go out
    // evict-first (streaming stores).
    const uint64_t keep_l2 = l2_policy_evict_last();
    auto issue = [&](int s, int p) {
        unsigned char* q = smem + s * Lay::kStage;
        const int k = k0 + p;
        mbar_arrive_expect_tx(&bar[s], p < planes ? Lay::kTx : Lay::kTxE);
        tma_load_3d_hint(q + 0 * Lay::kEBytes, &maps.ex, x0 - 4, y0 - 1, k, &bar[s], keep_l2);
        tma_load_3d_hint(q + 1 * Lay::kEBytes, &maps.ey, x0 - 4, y0 - 1, k, &bar[s], keep_l2);
        tma_load_3d_hint(q + 2 * Lay::kEBytes, &maps.ez, x0 - 4, y0 - 1, k, &bar[s], keep_l2);
        if (p < planes) {
            unsigned char* h = q + 3 * Lay::kEBytes;
            tma_load_3d(h + 0 * Lay::kHBytes, &maps.hx, x0 - 4, y0 - 1, k, &bar[s]);
            tma_load_3d(h + 1 * Lay::kHBytes, &maps.hy, x0 - 4, y0 - 1, k, &bar[s]);
            tma_load_3d(h + 2 * Lay::kHBytes, &maps.hz, x0 - 4, y0 - 1, k, &bar[s]);
            tma_load_3d(h + 3 * Lay::kHBytes, &maps.mat, x0, y0, k, &bar[s]);
        }
    };
    auto mat_of = [&](int s) -> uint8_t {
        return (smem + s * Lay::kStage + 3 * Lay::kEBytes + 3 * Lay::kHBytes)[tcell];
    };
    auto gslot = [&](int b, int q) -> float* { return gbuf + (b * 9 + q) * T + tid; };
    auto prefetch_gain = [&](int b, uint32_t cc) {
        cp_async_4(gslot(b, 0), f.px + cc);
        cp_async_4(gslot(b, 1), f.py + cc);
        cp_async_4(gslot(b, 2), f.pz + cc);
        cp_async_4(gslot(b, 3), f.jx + cc);
        cp_async_4(gslot(b, 4), f.jy + cc);
        cp_async_4(gslot(b, 5), f.jz + cc);
        cp_async_4(gslot(b, 6), f.n1 + cc);
        cp_async_4(gslot(b, 7), f.n2 + cc);
        cp_async_4(gslot(b, 8), f.n3 + cc);
    };

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        fence_barrier_init();
    }
    if (tid < 6 * NW) wfl[tid / NW][tid % NW] = 0.0f;
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < S && s < total; ++s) issue(s, s);
    int issued = min(S, total);   // planes issued into the ring so far
    bool block_fail = false;

    uint32_t c = valid ? (uint32_t)i + (uint32_t)nx * j + nxy * k0 : 0u;
    // H^{n+1/2} of plane k0-1 at this cell (zero below the first plane)
    float hx_km1 = 0.0f, hy_km1 = 0.0f;
    if (valid && k0 > 0) {
        const uint32_t cm = c - nxy;
        const ENb e = load_e_nbrs(a, i, j, k0 - 1, cm);
        float hx = __ldg(f.hx + cm), hy = __ldg(f.hy + cm), hz = __ldg(f.hz + cm);
        const PsiOut none{nullptr, nullptr, nullptr};
        if (pml_xy || plane_in_z_slab(a, k0 - 1)) h_compute_to<true, false>(a, i, j, k0 - 1, e, hx, hy, hz, none);
        else h_compute_to<false, false>(a, i, j, k0 - 1, e, hx, hy, hz, none);
        hx_km1 = hx;
        hy_km1 = hy;
    }

    // Edge work: threads tid < BX take the cell (x0 + tid, y0 - 1) of the
    // halo row, threads BX <= tid < BX + BY the cell (x0 - 1, y0 + tid - BX)
    // of the halo column; cells outside the grid hold H = 0.
    const bool row = tid < BX, col = !row && tid < BX + BY;
    const int hi = row ? x0 + tid : x0 - 1;
    const int hj = row ? y0 - 1 : y0 + (tid - BX);
    const bool halo = (row || col) && hi >= 0 && hj >= 0 && hi < nx && hj < ny;
    const int halo_e = row ? tid + 4 : (tid - BX + 1) * Lay::kEX + 3;
    const int halo_h = row ? tid + 4 : (tid - BX + 1) * Lay::kHX + 3;
    const int halo_n = row ? tid + 1 : (tid - BX + 1) * Lay::kNX;
    // Warp-uniform path choices (a path taken for cells it does not need
    // gives the same bits: the CPML code leaves cells outside the slabs
    // alone, and the flux terms of cells off the faces are zero): the CPML
    // code for the warp's own cells and for its halo cells where one of them
    // lies in an x or y slab (or the plane in a z slab), the flux terms where
    // one of its cells lies on an x or y face of the flux box (within the
    // box's z range) or the plane is a z face.
    const unsigned full = 0xffffffffu;
    const bool w_pml = __any_sync(full, pml_xy && valid && cell_in_xy_slab(a, i, j));
    const bool w_pml_halo = __any_sync(full, pml_xy && halo && cell_in_xy_slab(a, hi, hj));
    const bool w_xy = __any_sync(full, face && valid && cells_on_xy_face(a.flux, i, 1, j));
    const int own_e = (ty + 1) * Lay::kEX + tx + 4;
    const int own_h = (ty + 1) * Lay::kHX + tx + 4;
    const int own_n = (ty + 1) * Lay::kNX + tx + 1;
    constexpr int EW = Lay::kEBytes / 4, HW = Lay::kHBytes / 4, NN = Lay::kNW;

    bool fail = !mbar_wait_bounded(&bar[0], 0, kWaitLimit);
    bool pg = valid && gain_on && !fail && (mat_of(0) & 0x80);
    if (pg) prefetch_gain(0, c);
    cp_async_commit();
    // ring slots of planes p and p + 1, and the phase parity of plane p + 1
    int s = 0, s1 = 1 % S;
    uint32_t ph1 = (1 / S) & 1;
    for (int p = 0; p < planes; ++p) {
        const int k = k0 + p;
        cp_async_wait_all();   // this plane's gain values (own thread's copies)
        fail |= !mbar_wait_bounded(&bar[s1], ph1, kWaitLimit);
        bool ng = false;
        if (p + 1 < planes) {
            ng = valid && gain_on && !fail && (mat_of(s1) & 0x80);
            if (ng) prefetch_gain((p + 1) & 1, c + nxy);
        }
        cp_async_commit();
        const float* E0 = reinterpret_cast<const float*>(smem + s * Lay::kStage);
        const float* E1 = reinterpret_cast<const float*>(smem + s1 * Lay::kStage);
        const float* H0 = reinterpret_cast<const float*>(smem + s * Lay::kStage + 3 * Lay::kEBytes);
        const bool zpml = plane_in_z_slab(a, k);
        const bool pml = w_pml || zpml, pml_h = w_pml_halo || zpml;
        const bool fk = plane_has_flux(a.flux, face, w_xy, k);

        // 1. H^{n+1/2}: own cell, then the halo row / column
        float hx = 0.0f, hy = 0.0f, hz = 0.0f;
        if (valid && !fail) {
            ENb e;
            e.ex = E0[own_e];
            e.ey = E0[EW + own_e];
            e.ez = E0[2 * EW + own_e];
            e.ex_j1 = E0[own_e + Lay::kEX];
            e.ez_j1 = E0[2 * EW + own_e + Lay::kEX];
            e.ey_i1 = E0[EW + own_e + 1];
            e.ez_i1 = E0[2 * EW + own_e + 1];
            e.ex_k1 = E1[own_e];
            e.ey_k1 = E1[EW + own_e];
            hx = H0[own_h];
            hy = H0[HW + own_h];
            hz = H0[2 * HW + own_h];
            if (pml) h_compute_to<true, true>(a, i, j, k, e, hx, hy, hz, d.psi);
            else h_compute_to<false, true>(a, i, j, k, e, hx, hy, hz, d.psi);
            __stcs(d.hx + c, hx);
            __stcs(d.hy + c, hy);
            __stcs(d.hz + c, hz);
            // the CPML memories the E update reads after the barrier
            if (pml) prefetch_psi(a, i, j, k, 0);
        }
        hn[own_n] = hx;
        hn[NN + own_n] = hy;
        hn[2 * NN + own_n] = hz;
        if (row || col) {
            float qx = 0.0f, qy = 0.0f, qz = 0.0f;
            if (halo && !fail) {
                ENb e;
                e.ex = E0[halo_e];
                e.ey = E0[EW + halo_e];
                e.ez = E0[2 * EW + halo_e];
                e.ex_j1 = E0[halo_e + Lay::kEX];
                e.ez_j1 = E0[2 * EW + halo_e + Lay::kEX];
                e.ey_i1 = E0[EW + halo_e + 1];
                e.ez_i1 = E0[2 * EW + halo_e + 1];
                e.ex_k1 = E1[halo_e];
                e.ey_k1 = E1[EW + halo_e];
                qx = H0[halo_h];
                qy = H0[HW + halo_h];
                qz = H0[2 * HW + halo_h];
                const PsiOut none{nullptr, nullptr, nullptr};
                if (pml_h) h_compute_to<true, false>(a, hi, hj, k, e, qx, qy, qz, none);
                else h_compute_to<false, false>(a, hi, hj, k, e, qx, qy, qz, none);
            }
            hn[halo_n] = qx;
            hn[NN + halo_n] = qy;
            hn[2 * NN + halo_n] = qz;
        }

        // 2. J^{n+1/2}, P^{n+1} of a gain cell (time-n state only)
        const int b = p & 1;
        float jx = 0.f, jy = 0.f, jz = 0.f, n1 = 0.f, n2 = 0.f, n3 = 0.f;
        if (pg && !fail) {
            float px = *gslot(b, 0), py = *gslot(b, 1), pz = *gslot(b, 2);
            jx = *gslot(b, 3);
            jy = *gslot(b, 4);
            jz = *gslot(b, 5);
            n1 = *gslot(b, 6);
            n2 = *gslot(b, 7);
            n3 = *gslot(b, 8);
            lorentz_step(a.gain, c, n, E0[own_e], E0[EW + own_e], E0[2 * EW + own_e], n1, n2, jx,
                         jy, jz, px, py, pz);
            __stcs(f.px + c, px);
            __stcs(f.py + c, py);
            __stcs(f.pz + c, pz);
            __stcs(f.jx + c, jx);
            __stcs(f.jy + c, jy);
            __stcs(f.jz + c, jz);
        }
        __syncthreads();   // the H tile is complete

        // 3. E^{n+1}, N^{n+1}, face flux
        float fl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid && !fail) {
            HNb h;
            h.hx = hx;
            h.hy = hy;
            h.hz = hz;
            h.hy_i = hn[NN + own_n - 1];
            h.hz_i = hn[2 * NN + own_n - 1];
            h.hx_j = hn[own_n - Lay::kNX];
            h.hz_j = hn[2 * NN + own_n - Lay::kNX];
            h.hx_k = hx_km1;
            h.hy_k = hy_km1;
            const uint8_t m = mat_of(s);
            const float ex0 = E0[own_e], ey0 = E0[EW + own_e], ez0 = E0[2 * EW + own_e];
            float ex1, ey1, ez1;
            if (fk)
                e_compute_to<true, true>(a, i, j, k, c, h, m, ex0, ey0, ez0, pg, jx, jy, jz, n1, n2,
                                         n3, n, fl, ex1, ey1, ez1, d.psi);
            else if (pml)
                e_compute_to<false, true>(a, i, j, k, c, h, m, ex0, ey0, ez0, pg, jx, jy, jz, n1, n2,
                                          n3, n, fl, ex1, ey1, ez1, d.psi);
            else
                e_compute_to<false, false>(a, i, j, k, c, h, m, ex0, ey0, ez0, pg, jx, jy, jz, n1,
                                           n2, n3, n, fl, ex1, ey1, ez1, d.psi);
            __stcs(d.ex + c, ex1);
            __stcs(d.ey + c, ey1);
            __stcs(d.ez + c, ez1);
            if (pg) {
                __stcs(f.n1 + c, n1);
                __stcs(f.n2 + c, n2);
                __stcs(f.n3 + c, n3);
            }
            hx_km1 = hx;
            hy_km1 = hy;
            // the CPML memories the next plane's H update reads
            if (p + 1 < planes && (w_pml || plane_in_z_slab(a, k + 1))) prefetch_psi(a, i, j, k + 1, 2);
        }
        if (fk) {
            // this plane's flux terms: warp sums, added to the warp's partials
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                float v = fl[q];
                if (__any_sync(full, v != 0.0f)) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
                    if ((tid & 31) == 0) wfl[q][tid >> 5] += v;
                }
            }
        }
        // ring slot s and the H tile are free again; the barrier also ORs the
        // threads' wait verdicts, so every thread sees the same block_fail
        block_fail = __syncthreads_or(fail);
        if (block_fail) break;   // issue nothing more; drained below
        if (p + S < total) {
            if (tid == 0) issue(s, p + S);
            issued = p + S + 1;
        }
        pg = ng;
        c += nxy;
        s = s1;
        s1 = (s1 + 1 == S) ? 0 : s1 + 1;
        if (s1 == 0) ph1 ^= 1u;
    }
    cp_async_wait_all();
    if (block_fail) {
        // A wait gave up: record it, then give the copies still in flight a
        // bounded chance to land before the block's shared memory is released.
        if (tid == 0) atomicOr(a.err, 1);
        drain_ring(bar, S, issued, kWaitLimit);
    }
    if (face && (tid & 31) == 0) {
        const unsigned slot = warp_slot();
#pragma unroll
        for (int q = 0; q < 6; ++q)
            if (wfl[q][tid >> 5] != 0.0f)
                atomicAdd(a.flux.acc + q * kFluxSlots + (slot % kFluxSlots), (double)wfl[q][tid >> 5]);
    }
    finish_step(a, d.sample);
}

template <int BX, int BY>
static void launch_fused(const StepArgs& a, const DevPing& d, int kz, const TmaFusedMaps& maps,
                         cudaStream_t s) {
    const int smem = FusedLayout<BX, BY>::smem_bytes(kTmaStages);
    static bool attr_set = false;   // per instantiation, once per process
    if (!attr_set) {
        cudaFuncSetAttribute(k_step_fused<BX, BY, kTmaStages>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr_set = true;
    }
    dim3 grid((a.g.nx + BX - 1) / BX, (a.g.ny + BY - 1) / BY, fused_z_blocks(a.g.nz, kz));
    k_step_fused<BX, BY, kTmaStages><<<grid, dim3(BX, BY, 1), smem, s>>>(a, d, maps, kz);
}

bool fused_tile_supported(int bx, int by) {
    return (bx == 32 || bx == 64) && (by == 4 || by == 8);
}

bool encode_fused(const StepArgs& a, int bx, int by, TmaFusedMaps* out) {
    if (!tma_e_supported(a) || !fused_tile_supported(bx, by)) return false;
    const DevFields& f = a.f;
    const CUtensorMapDataType F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    return encode_box(&out->ex, F32, f.ex, 4, a.g, bx + 8, by + 2) &&
           encode_box(&out->ey, F32, f.ey, 4, a.g, bx + 8, by + 2) &&
           encode_box(&out->ez, F32, f.ez, 4, a.g, bx + 8, by + 2) &&
           encode_box(&out->hx, F32, f.hx, 4, a.g, bx + 4, by + 1) &&
           encode_box(&out->hy, F32, f.hy, 4, a.g, bx + 4, by + 1) &&
           encode_box(&out->hz, F32, f.hz, 4, a.g, bx + 4, by + 1) &&
           encode_box(&out->mat, CU_TENSOR_MAP_DATA_TYPE_UINT8, f.mat, 1, a.g, bx, by);
}

void launch_fused_step(const StepArgs& a, const DevPing& d, const PassTune& t,
                       const TmaFusedMaps& maps, cudaStream_t s) {
    const int bx = t.block.x, by = t.block.y;
    if (bx == 32 && by == 4) launch_fused<32, 4>(a, d, t.kz, maps, s);
    else if (bx == 32 && by == 8) launch_fused<32, 8>(a, d, t.kz, maps, s);
    else if (bx == 64 && by == 4) launch_fused<64, 4>(a, d, t.kz, maps, s);
    else if (bx == 64 && by == 8) launch_fused<64, 8>(a, d, t.kz, maps, s);
}

}  // namespace mb
