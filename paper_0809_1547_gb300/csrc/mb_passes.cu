// Field-pass kernels of the Maxwell–Bloch FDTD step and their launchers.
//
// One time step is two launches:
//   k_hg_*  the H half-step over every cell, and, in blocks of their own, the
//           Lorentz / Langevin update of the gain cells (a static list), so
//           the Philox and Box–Muller work runs in full warps;
//   k_e_*   the E update of every cell with the fresh J^{n+1/2}, the
//           population update of gain cells and the face flux; its last
//           block to finish increments the step counter.
// Both are memory-bound stencils (no tensor cores: nothing here is a dense
// contraction).  Variants: 3-D tiles with one thread per cell, or 2-D tiles
// whose threads walk kz planes of their column with the neighbour plane in
// registers.  Every variant composes the same per-cell helpers, so all of
// them produce the same bits.
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

__device__ __forceinline__ void gain_block(const StepArgs& a, unsigned gidx, int q, long long n) {
    const int T = blockDim.x * blockDim.y * blockDim.z;
    const uint32_t base = gidx * (uint32_t)q;
    for (int r = linear_tid(); r < q; r += T) {
        const uint32_t e = base + (uint32_t)r;
        if (e < a.glist.count) gain_cell_step(a, __ldg(a.glist.cell + e), n);
    }
}

// Does the tile [i0, i0+bx) x [j0, j0+by) touch an x or y CPML slab?
__device__ __forceinline__ bool tile_in_xy_slab(const StepArgs& a, int i0, int bx, int j0, int by) {
    const int L = a.pml.L;
    return L > 0 && (i0 < L || i0 + bx > a.g.nx - L || j0 < L || j0 + by > a.g.ny - L);
}

__device__ __forceinline__ bool plane_in_z_slab(const StepArgs& a, int k) {
    const int L = a.pml.L;
    return L > 0 && (k < L || k >= a.g.nz - L);
}

// ------------------------------------------------------ H + gain launches

__global__ void __launch_bounds__(512) k_hg_3d(StepArgs a, HGLayout lay) {
    const long long n = a.step_ctr[0];
    unsigned idx;
    if (hg_block_kind(lay, blockIdx.x, idx)) {
        gain_block(a, idx, lay.q, n);
        return;
    }
    const int bx = idx % lay.gx, by = (idx / lay.gx) % lay.gy, bz = idx / (lay.gx * lay.gy);
    const int i = bx * blockDim.x + threadIdx.x;
    const int j = by * blockDim.y + threadIdx.y;
    const int k = bz * blockDim.z + threadIdx.z;
    if (i >= a.g.nx || j >= a.g.ny || k >= a.g.nz) return;
    const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
    const ENb e = load_e_nbrs(a, i, j, k, c);
    const int k0 = bz * blockDim.z;
    const bool pml = tile_in_xy_slab(a, bx * blockDim.x, blockDim.x, by * blockDim.y, blockDim.y) ||
                     plane_in_z_slab(a, k0) || plane_in_z_slab(a, k0 + blockDim.z - 1);
    if (pml) h_core<true>(a, i, j, k, c, e);
    else h_core<false>(a, i, j, k, c, e);
}

__global__ void __launch_bounds__(512) k_hg_zmarch(StepArgs a, HGLayout lay, int kz) {
    const long long n = a.step_ctr[0];
    unsigned idx;
    if (hg_block_kind(lay, blockIdx.x, idx)) {
        gain_block(a, idx, lay.q, n);
        return;
    }
    const int bx = idx % lay.gx, by = (idx / lay.gx) % lay.gy, bz = idx / (lay.gx * lay.gy);
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
    for (int k = k0; k < k1; ++k, c += nxy) {
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
        ex_c = e.ex_k1;
        ey_c = e.ey_k1;
    }
}

// ------------------------------------------------------------ E launches

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

// The last block of the E launch to finish advances the step counter.  No
// block waits for another: each one only counts itself out.
__device__ __forceinline__ void finish_step(const StepArgs& a) {
    __syncthreads();
    if (linear_tid() == 0) {
        __threadfence();
        const unsigned long long nb = (unsigned long long)gridDim.x * gridDim.y * gridDim.z;
        const unsigned long long t = atomicAdd((unsigned long long*)(a.step_ctr + 1), 1ULL);
        if (t == nb - 1) {
            atomicExch((unsigned long long*)(a.step_ctr + 1), 0ULL);
            atomicAdd((unsigned long long*)a.step_ctr, 1ULL);
        }
    }
}

__global__ void __launch_bounds__(512, 2) k_e_3d(StepArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z * blockDim.z + threadIdx.z;
    const long long n = a.step_ctr[0];
    const bool valid = i < a.g.nx && j < a.g.ny && k < a.g.nz;
    const int i0 = blockIdx.x * blockDim.x, j0 = blockIdx.y * blockDim.y, k0 = blockIdx.z * blockDim.z;
    const bool face = tile_on_face(a.flux, i0, i0 + blockDim.x, j0, j0 + blockDim.y, k0, k0 + blockDim.z);
    const bool pml = tile_in_xy_slab(a, i0, blockDim.x, j0, blockDim.y) || plane_in_z_slab(a, k0) ||
                     plane_in_z_slab(a, k0 + blockDim.z - 1);
    float fl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
        const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
        const HNb h = load_h_nbrs(a, i, j, k, c);
        if (face) e_core<true, true>(a, i, j, k, c, h, n, fl);
        else if (pml) e_core<false, true>(a, i, j, k, c, h, n, fl);
        else e_core<false, false>(a, i, j, k, c, h, n, fl);
    }
    if (face) flux_warp_reduce(a.flux, fl, warp_slot());
    finish_step(a);
}

// Walk of one column (i, j) over planes [k0, k1).  FACE: the block holds
// face-plane cells (flux terms summed into fl over the walk); PML_XY: the
// tile touches an x or y CPML slab (else only z-slab planes take the CPML
// code).
template <bool FACE, bool PML_XY>
__device__ __forceinline__ void e_walk(const StepArgs& a, int i, int j, int k0, int k1, long long n,
                                       float fl[6]) {
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
        if (FACE || PML_XY) e_core<FACE, true>(a, i, j, k, c, h, n, fl);
        else if (plane_in_z_slab(a, k)) e_core<false, true>(a, i, j, k, c, h, n, fl);
        else e_core<false, false>(a, i, j, k, c, h, n, fl);
        hx_km1 = h.hx;
        hy_km1 = h.hy;
    }
}

__global__ void __launch_bounds__(512, 2) k_e_zmarch(StepArgs a, int kz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int nz = a.g.nz;
    const bool valid = i < a.g.nx && j < a.g.ny;   // no early exit: warp-wide flux reduction
    const long long n = a.step_ctr[0];
    const int k0 = blockIdx.z * kz;
    const int k1 = min(nz, k0 + kz);
    const int i0 = blockIdx.x * blockDim.x, j0 = blockIdx.y * blockDim.y;
    const bool face = tile_on_face(a.flux, i0, i0 + blockDim.x, j0, j0 + blockDim.y, k0, k1);
    const bool pml_xy = tile_in_xy_slab(a, i0, blockDim.x, j0, blockDim.y);
    if (face) {
        float fl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid) e_walk<true, true>(a, i, j, k0, k1, n, fl);
        flux_warp_reduce(a.flux, fl, warp_slot());
    } else if (valid) {
        float* none = nullptr;
        if (pml_xy) e_walk<false, true>(a, i, j, k0, k1, n, none);
        else e_walk<false, false>(a, i, j, k0, k1, n, none);
    }
    finish_step(a);
}

// -------------------------------------------------------------- launchers

HGLayout hg_layout(const StepArgs& a, const PassTune& t) {
    HGLayout L;
    L.gx = (a.g.nx + t.block.x - 1) / t.block.x;
    L.gy = (a.g.ny + t.block.y - 1) / t.block.y;
    const int zdiv = t.variant == kVariantZmarch ? t.kz : (int)t.block.z;
    L.gz = (a.g.nz + zdiv - 1) / zdiv;
    L.nH = L.gx * L.gy * L.gz;
    const int threads = t.block.x * t.block.y * (t.variant == kVariantZmarch ? 1 : t.block.z);
    L.q = threads * 4;
    L.nG = (a.gain.on && a.glist.count) ? (int)((a.glist.count + L.q - 1) / L.q) : 0;
    return L;
}

void launch_h_pass(const StepArgs& a, const PassTune& t, cudaStream_t s) {
    const HGLayout L = hg_layout(a, t);
    const unsigned blocks = (unsigned)(L.nH + L.nG);
    if (t.variant == kVariantZmarch) {
        k_hg_zmarch<<<blocks, dim3(t.block.x, t.block.y, 1), 0, s>>>(a, L, t.kz);
    } else {
        k_hg_3d<<<blocks, t.block, 0, s>>>(a, L);
    }
}

void launch_e_pass(const StepArgs& a, const PassTune& t, cudaStream_t s) {
    if (t.variant == kVariantZmarch) {
        dim3 grid((a.g.nx + t.block.x - 1) / t.block.x, (a.g.ny + t.block.y - 1) / t.block.y,
                  (a.g.nz + t.kz - 1) / t.kz);
        k_e_zmarch<<<grid, dim3(t.block.x, t.block.y, 1), 0, s>>>(a, t.kz);
    } else {
        dim3 grid((a.g.nx + t.block.x - 1) / t.block.x, (a.g.ny + t.block.y - 1) / t.block.y,
                  (a.g.nz + t.block.z - 1) / t.block.z);
        k_e_3d<<<grid, t.block, 0, s>>>(a);
    }
}

}  // namespace mb
