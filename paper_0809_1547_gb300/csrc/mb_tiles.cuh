// Per-tile device functions shared by the step's launches (plain passes,
// batched ensemble): the gain-list blocks, the z-walking H and E tiles, the
// face-flux slots and the step counter.  Every launch composes these, so the
// arithmetic of a cell is the same in all of them.
#pragma once

#include "mb_host.h"

namespace mb {

// Block b of the H + gain grid is a gain block (returns true, idx = its
// index) or an H block (returns false, idx = its index).  Gain blocks are
// spread evenly through the grid so both kinds advance through the domain
// together and the gain blocks' E^n reads find the H blocks' lines in L2.
__device__ __forceinline__ bool hg_block_kind(const HGLayout& L, unsigned b, unsigned& idx) {
    const unsigned long long tot = (unsigned long long)L.nH + L.nG;
    const unsigned g0 = (unsigned)((unsigned long long)b * L.nG / tot);
    const unsigned g1 = (unsigned)((unsigned long long)(b + 1) * L.nG / tot);
    if (g1 > g0) {
        idx = g0;
        return true;
    }
    idx = b - g0;
    return false;
}

__device__ __forceinline__ int linear_tid() {
    return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}

// A gain block advances q = PER * threads consecutive entries of the gain
// list; each thread loads all its PER cells before computing any, so that
// several cells' loads are in flight at once.
template <int PER = kGainPerThread>
__device__ __forceinline__ void gain_block(const StepArgs& a, unsigned gidx, int q, long long n) {
    const int T = blockDim.x * blockDim.y * blockDim.z;
    const uint32_t base = gidx * (uint32_t)q + (uint32_t)linear_tid();
    const DevFields& f = a.f;
    uint32_t cs[PER];
    bool ok[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const uint32_t e = base + (uint32_t)(r * T);
        ok[r] = e < a.glist.count;
        cs[r] = ok[r] ? __ldg(a.glist.cell + e) : 0u;
    }
    float ex[PER], ey[PER], ez[PER], n1[PER],
        n2[PER], px[PER], py[PER], pz[PER],
        jx[PER], jy[PER], jz[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        if (!ok[r]) continue;
        const uint32_t c = cs[r];
        ex[r] = __ldg(f.ex + c);
        ey[r] = __ldg(f.ey + c);
        ez[r] = __ldg(f.ez + c);
        n1[r] = f.n1[c];
        n2[r] = f.n2[c];
        px[r] = f.px[c];
        py[r] = f.py[c];
        pz[r] = f.pz[c];
        jx[r] = f.jx[c];
        jy[r] = f.jy[c];
        jz[r] = f.jz[c];
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        if (!ok[r]) continue;
        const uint32_t c = cs[r];
        lorentz_step(a.gain, c, n, ex[r], ey[r], ez[r], n1[r], n2[r], jx[r], jy[r], jz[r], px[r],
                     py[r], pz[r]);
        f.jx[c] = jx[r];
        f.jy[c] = jy[r];
        f.jz[c] = jz[r];
        f.px[c] = px[r];
        f.py[c] = py[r];
        f.pz[c] = pz[r];
    }
}

// Does the tile [i0, i0+bx) x [j0, j0+by) touch an x or y CPML slab?
__device__ __forceinline__ bool tile_in_xy_slab(const StepArgs& a, int i0, int bx, int j0, int by) {
    const int L = a.pml.L;
    return L > 0 && (i0 < L || i0 + bx > a.g.nx - L || j0 < L || j0 + by > a.g.ny - L);
}

__device__ __forceinline__ bool plane_in_z_slab(const StepArgs& a, int k) {
    return a.pml.L > 0 && (k < a.pml.zlo || k >= a.pml.zhi);
}

// Cell (i, j) lies in an x or y CPML slab.
__device__ __forceinline__ bool cell_in_xy_slab(const StepArgs& a, int i, int j) {
    const int L = a.pml.L;
    return L > 0 && (i < L || i >= a.g.nx - L || j < L || j >= a.g.ny - L);
}

// Cells (i0 .. i0+w-1, j) can hold terms of an x or y face of the flux box
// (on some plane of the box's z range).
__device__ __forceinline__ bool cells_on_xy_face(const DevFlux& F, int i0, int w, int j) {
    if (!F.on) return false;
    const bool xf = ((F.plo[0] >= i0 && F.plo[0] < i0 + w) || (F.phi[0] >= i0 && F.phi[0] < i0 + w)) &&
                    j >= F.r0[1] && j < F.r1[1];
    const bool yf = (j == F.plo[1] || j == F.phi[1]) && i0 + w > F.r0[0] && i0 < F.r1[0];
    return xf || yf;
}

// Plane k of a block holding face cells (face) needs the flux terms in a
// warp: the warp holds cells of an x or y face (w_xy) and k lies in the
// box's z range, or k is a z face.  Elsewhere every term is zero.
__device__ __forceinline__ bool plane_has_flux(const DevFlux& F, bool face, bool w_xy, int k) {
    return face && ((w_xy && k >= F.r0[2] && k < F.r1[2]) || k == F.plo[2] || k == F.phi[2]);
}

// ------------------------------------------------------------ H tiles

// H walk of tile (bx, by, bz): a 2-D block over (x, y), kz planes per thread.
__device__ __forceinline__ void h_tile_zmarch(const StepArgs& a, int bx, int by, int bz, int kz) {
    const int i = bx * blockDim.x + threadIdx.x;
    const int j = by * blockDim.y + threadIdx.y;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    if (i >= nx || j >= ny) return;
    const int k0 = bz * kz;
    const int k1 = min(nz, k0 + kz);
    const uint32_t nxy = a.g.nxy;
    const float* __restrict__ Ex = a.f.ex;
    const float* __restrict__ Ey = a.f.ey;
    const float* __restrict__ Ez = a.f.ez;
    const bool xi = i + 1 < nx, yj = j + 1 < ny;
    const bool pml_xy = tile_in_xy_slab(a, bx * blockDim.x, blockDim.x, by * blockDim.y, blockDim.y);
    uint32_t c = (uint32_t)i + (uint32_t)nx * j + nxy * k0;
    float ex_c = __ldg(Ex + c), ey_c = __ldg(Ey + c);
    int k = k0;
    // two planes per iteration: all loads of both are issued before either update
    for (; k + 1 < k1; k += 2, c += 2 * nxy) {
        ENb e0, e1;
        const bool zk = k + 2 < nz;
        e0.ex = ex_c;
        e0.ey = ey_c;
        e0.ez = __ldg(Ez + c);
        e0.ex_k1 = __ldg(Ex + c + nxy);
        e0.ey_k1 = __ldg(Ey + c + nxy);
        e0.ex_j1 = yj ? __ldg(Ex + c + nx) : 0.0f;
        e0.ey_i1 = xi ? __ldg(Ey + c + 1) : 0.0f;
        e0.ez_i1 = xi ? __ldg(Ez + c + 1) : 0.0f;
        e0.ez_j1 = yj ? __ldg(Ez + c + nx) : 0.0f;
        const uint32_t c1 = c + nxy;
        e1.ex = e0.ex_k1;
        e1.ey = e0.ey_k1;
        e1.ez = __ldg(Ez + c1);
        e1.ex_k1 = zk ? __ldg(Ex + c1 + nxy) : 0.0f;
        e1.ey_k1 = zk ? __ldg(Ey + c1 + nxy) : 0.0f;
        e1.ex_j1 = yj ? __ldg(Ex + c1 + nx) : 0.0f;
        e1.ey_i1 = xi ? __ldg(Ey + c1 + 1) : 0.0f;
        e1.ez_i1 = xi ? __ldg(Ez + c1 + 1) : 0.0f;
        e1.ez_j1 = yj ? __ldg(Ez + c1 + nx) : 0.0f;
        if (pml_xy || plane_in_z_slab(a, k)) h_core<true>(a, i, j, k, c, e0);
        else h_core<false>(a, i, j, k, c, e0);
        if (pml_xy || plane_in_z_slab(a, k + 1)) h_core<true>(a, i, j, k + 1, c1, e1);
        else h_core<false>(a, i, j, k + 1, c1, e1);
        ex_c = e1.ex_k1;
        ey_c = e1.ey_k1;
    }
    if (k < k1) {
        ENb e;
        const bool zk = k + 1 < nz;
        e.ex = ex_c;
        e.ey = ey_c;
        e.ez = __ldg(Ez + c);
        e.ex_k1 = zk ? __ldg(Ex + c + nxy) : 0.0f;
        e.ey_k1 = zk ? __ldg(Ey + c + nxy) : 0.0f;
        e.ex_j1 = yj ? __ldg(Ex + c + nx) : 0.0f;
        e.ey_i1 = xi ? __ldg(Ey + c + 1) : 0.0f;
        e.ez_i1 = xi ? __ldg(Ez + c + 1) : 0.0f;
        e.ez_j1 = yj ? __ldg(Ez + c + nx) : 0.0f;
        if (pml_xy || plane_in_z_slab(a, k)) h_core<true>(a, i, j, k, c, e);
        else h_core<false>(a, i, j, k, c, e);
    }
}

// ------------------------------------------------------------ E tiles


// Blocks whose cell range contains a face plane reduce the flux (uniform).
__device__ __forceinline__ bool tile_on_face(const DevFlux& F, int i0, int i1, int j0, int j1,
                                             int k0, int k1) {
    if (!F.on) return false;
    return (F.plo[0] >= i0 && F.plo[0] < i1) || (F.phi[0] >= i0 && F.phi[0] < i1) ||
           (F.plo[1] >= j0 && F.plo[1] < j1) || (F.phi[1] >= j0 && F.phi[1] < j1) ||
           (F.plo[2] >= k0 && F.plo[2] < k1) || (F.phi[2] >= k0 && F.phi[2] < k1);
}

__device__ __forceinline__ unsigned warp_slot() {
    const unsigned b = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    return b * 7u + (unsigned)(linear_tid() >> 5);
}

// The last block of the E launch to finish advances the step counter (and
// stores the new count in *sample when given).  No block waits for another:
// each one only counts itself out.
__device__ __forceinline__ void finish_step(const StepArgs& a, long long* sample = nullptr) {
    __syncthreads();
    if (linear_tid() == 0) {
        __threadfence();
        const unsigned long long nb = (unsigned long long)gridDim.x * gridDim.y * gridDim.z;
        const unsigned long long t = atomicAdd((unsigned long long*)(a.step_ctr + 1), 1ULL);
        if (t == nb - 1) {
            atomicExch((unsigned long long*)(a.step_ctr + 1), 0ULL);
            const unsigned long long prev = atomicAdd((unsigned long long*)a.step_ctr, 1ULL);
            if (sample) *sample = (long long)prev + 1;
        }
    }
}

// Walk of one column (i, j) over planes [k0, k1).  FACE: the block holds
// face-plane cells (flux terms summed into fl over the walk, taken on the
// planes plane_has_flux names; w_xy is warp-uniform); PML_XY: the tile
// touches an x or y CPML slab (else only z-slab planes take the CPML code).
template <bool FACE, bool PML_XY>
__device__ __forceinline__ void e_walk(const StepArgs& a, int i, int j, int k0, int k1, long long n,
                                       float fl[6], bool w_xy = false) {
    const int nx = a.g.nx;
    const uint32_t nxy = a.g.nxy;
    const float* __restrict__ Hx = a.f.hx;
    const float* __restrict__ Hy = a.f.hy;
    const float* __restrict__ Hz = a.f.hz;
    uint32_t c = (uint32_t)i + (uint32_t)nx * j + nxy * k0;
    float hx_km1 = 0.0f, hy_km1 = 0.0f;
    if (k0 > 0) {
        hx_km1 = __ldg(Hx + c - nxy);
        hy_km1 = __ldg(Hy + c - nxy);
    }
    for (int k = k0; k < k1; ++k, c += nxy) {
        HNb h;
        h.hx = __ldg(Hx + c);
        h.hy = __ldg(Hy + c);
        h.hz = __ldg(Hz + c);
        h.hx_k = hx_km1;
        h.hy_k = hy_km1;
        h.hx_j = (j > 0) ? __ldg(Hx + c - nx) : 0.0f;
        h.hz_j = (j > 0) ? __ldg(Hz + c - nx) : 0.0f;
        h.hy_i = (i > 0) ? __ldg(Hy + c - 1) : 0.0f;
        h.hz_i = (i > 0) ? __ldg(Hz + c - 1) : 0.0f;
        if (FACE || PML_XY) e_core<FACE, true>(a, i, j, k, c, h, n, fl,
                                               !FACE || plane_has_flux(a.flux, true, w_xy, k));
        else if (plane_in_z_slab(a, k)) e_core<false, true>(a, i, j, k, c, h, n, fl);
        else e_core<false, false>(a, i, j, k, c, h, n, fl);
        hx_km1 = h.hx;
        hy_km1 = h.hy;
    }
}

// E walk of tile (bx, by, bz) for step n (flux of face tiles included).
// Every thread of the block must call it (warp-wide flux reduction).
__device__ __forceinline__ void e_tile_zmarch(const StepArgs& a, int bx, int by, int bz, int kz,
                                              long long n, unsigned slot) {
    const int i = bx * blockDim.x + threadIdx.x;
    const int j = by * blockDim.y + threadIdx.y;
    const int nz = a.g.nz;
    const bool valid = i < a.g.nx && j < a.g.ny;
    const int k0 = bz * kz;
    const int k1 = min(nz, k0 + kz);
    const int i0 = bx * blockDim.x, j0 = by * blockDim.y;
    const bool face = tile_on_face(a.flux, i0, i0 + blockDim.x, j0, j0 + blockDim.y, k0, k1);
    const bool pml_xy = tile_in_xy_slab(a, i0, blockDim.x, j0, blockDim.y);
    if (face) {
        float fl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const bool w_xy = __any_sync(0xffffffffu, valid && cells_on_xy_face(a.flux, i, 1, j));
        if (valid) e_walk<true, true>(a, i, j, k0, k1, n, fl, w_xy);
        flux_warp_reduce(a.flux, fl, slot);
    } else if (valid) {
        float* none = nullptr;
        if (pml_xy) e_walk<false, true>(a, i, j, k0, k1, n, none);
        else e_walk<false, false>(a, i, j, k0, k1, n, none);
    }
}

}  // namespace mb
