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
#include "mb_tiles.cuh"
#include "mb_tma.cuh"

#include <cudaTypedefs.h>

namespace mb {
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
    h_tile_zmarch(a, idx % lay.gx, (idx / lay.gx) % lay.gy, idx / (lay.gx * lay.gy), kz);
}

// ------------------------------------------------------------ E launches

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

__global__ void __launch_bounds__(512, 2) k_e_zmarch(StepArgs a, int kz) {
    const long long n = a.step_ctr[0];
    e_tile_zmarch(a, blockIdx.x, blockIdx.y, blockIdx.z, kz, n, warp_slot());
    finish_step(a);
}

// ----------------------------------------------- quad-vectorised z-walks
// Each thread owns a quad of 4 consecutive x-cells (n_x % 4 == 0, so quads
// are 16-byte aligned) and moves them with 16-byte loads and stores, which
// stream at the full HBM rate where 4-byte accesses do not.  Warps lie along
// x: the +x (-x) neighbour of a quad's last (first) cell is the next
// (previous) lane's first (last) element, exchanged by shuffle; lane 31
// (lane 0) reads it from memory.  Lanes past the grid edge still take part
// in the shuffles with zeros.

__device__ __forceinline__ float4 ldg4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float& el(float4& v, int q) { return reinterpret_cast<float*>(&v)[q]; }
__device__ __forceinline__ float elc(const float4& v, int q) {
    return reinterpret_cast<const float*>(&v)[q];
}

__global__ void __launch_bounds__(256) k_hg_vec(StepArgs a, HGLayout lay, int kz) {
    const long long n = a.step_ctr[0];
    unsigned idx;
    if (hg_block_kind(lay, blockIdx.x, idx)) {
        gain_block(a, idx, lay.q, n);
        return;
    }
    const unsigned full = 0xffffffffu;
    const int bx = idx % lay.gx, by = (idx / lay.gx) % lay.gy, bz = idx / (lay.gx * lay.gy);
    const int lane = threadIdx.x & 31;
    const int i0 = 4 * (bx * blockDim.x + threadIdx.x);
    const int j = by * blockDim.y + threadIdx.y;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const bool valid = i0 < nx && j < ny;
    const bool yj = j + 1 < ny;
    const int k0 = bz * kz;
    const int k1 = min(nz, k0 + kz);
    const uint32_t nxy = a.g.nxy;
    const DevFields& f = a.f;
    const bool pml_xy = tile_in_xy_slab(a, 4 * bx * blockDim.x, 4 * blockDim.x, by * blockDim.y, blockDim.y);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t c = valid ? (uint32_t)i0 + (uint32_t)nx * j + nxy * k0 : 0u;
    float4 ex = valid ? ldg4(f.ex + c) : zero, ey = valid ? ldg4(f.ey + c) : zero;
    for (int k = k0; k < k1; ++k, c += nxy) {
        const bool zk = k + 1 < nz;
        const float4 ez = valid ? ldg4(f.ez + c) : zero;
        const float4 exk = (valid && zk) ? ldg4(f.ex + c + nxy) : zero;
        const float4 eyk = (valid && zk) ? ldg4(f.ey + c + nxy) : zero;
        const float4 exj = (valid && yj) ? ldg4(f.ex + c + nx) : zero;
        const float4 ezj = (valid && yj) ? ldg4(f.ez + c + nx) : zero;
        float ey_n = __shfl_down_sync(full, ey.x, 1);
        float ez_n = __shfl_down_sync(full, ez.x, 1);
        const bool xn = i0 + 4 < nx;
        if (lane == 31) {
            ey_n = (valid && xn) ? __ldg(f.ey + c + 4) : 0.0f;
            ez_n = (valid && xn) ? __ldg(f.ez + c + 4) : 0.0f;
        } else if (!xn) {
            ey_n = 0.0f;
            ez_n = 0.0f;
        }
        if (valid) {
            float4 hx = ld4(f.hx + c), hy = ld4(f.hy + c), hz = ld4(f.hz + c);
            const bool pml = pml_xy || plane_in_z_slab(a, k);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ENb e;
                e.ex = elc(ex, q);
                e.ey = elc(ey, q);
                e.ez = elc(ez, q);
                e.ex_j1 = elc(exj, q);
                e.ex_k1 = elc(exk, q);
                e.ey_i1 = q < 3 ? elc(ey, q + 1) : ey_n;
                e.ey_k1 = elc(eyk, q);
                e.ez_i1 = q < 3 ? elc(ez, q + 1) : ez_n;
                e.ez_j1 = elc(ezj, q);
                if (pml) h_compute<true>(a, i0 + q, j, k, e, el(hx, q), el(hy, q), el(hz, q));
                else h_compute<false>(a, i0 + q, j, k, e, el(hx, q), el(hy, q), el(hz, q));
            }
            st4(f.hx + c, hx);
            st4(f.hy + c, hy);
            st4(f.hz + c, hz);
        }
        ex = exk;
        ey = eyk;
    }
}

// The four cells of one quad: E^{n+1} into ex1..ez1, populations in place.
template <bool FACE, bool PML>
__device__ __forceinline__ void e_quad(const StepArgs& a, int i0, int j, int k, uint32_t c,
                                       const float4& hx, const float4& hy, const float4& hz,
                                       const float4& hxj, const float4& hzj, const float4& hxk,
                                       const float4& hyk, float hy_p, float hz_p, const float4& ex,
                                       const float4& ey, const float4& ez, uint32_t m4,
                                       const float4& jx, const float4& jy, const float4& jz,
                                       float4& n1, float4& n2, float4& n3, long long n, float fl[6],
                                       float4& ex1, float4& ey1, float4& ez1) {
    const bool gain_on = a.gain.on;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        HNb h;
        h.hx = elc(hx, q);
        h.hy = elc(hy, q);
        h.hz = elc(hz, q);
        h.hx_j = elc(hxj, q);
        h.hx_k = elc(hxk, q);
        h.hy_i = q > 0 ? elc(hy, q - 1) : hy_p;
        h.hy_k = elc(hyk, q);
        h.hz_i = q > 0 ? elc(hz, q - 1) : hz_p;
        h.hz_j = elc(hzj, q);
        const uint8_t m = (uint8_t)(m4 >> (8 * q));
        const bool g = gain_on && (m & 0x80);
        e_compute<FACE, PML>(a, i0 + q, j, k, c + q, h, m, elc(ex, q), elc(ey, q), elc(ez, q), g,
                             g ? elc(jx, q) : 0.0f, g ? elc(jy, q) : 0.0f, g ? elc(jz, q) : 0.0f,
                             el(n1, q), el(n2, q), el(n3, q), n, fl, el(ex1, q), el(ey1, q),
                             el(ez1, q));
    }
}

template <bool FACE>
__device__ __forceinline__ void e_vec_walk(const StepArgs& a, int i0, int j, int k0, int k1, bool valid,
                                           bool pml_xy, long long n, float fl[6], bool w_xy) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int nx = a.g.nx;
    const uint32_t nxy = a.g.nxy;
    const DevFields& f = a.f;
    const bool gain_on = a.gain.on;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t c = valid ? (uint32_t)i0 + (uint32_t)nx * j + nxy * k0 : 0u;
    float4 hxk = (valid && k0 > 0) ? ldg4(f.hx + c - nxy) : zero;
    float4 hyk = (valid && k0 > 0) ? ldg4(f.hy + c - nxy) : zero;
    for (int k = k0; k < k1; ++k, c += nxy) {
        const float4 hx = valid ? ldg4(f.hx + c) : zero;
        const float4 hy = valid ? ldg4(f.hy + c) : zero;
        const float4 hz = valid ? ldg4(f.hz + c) : zero;
        const float4 hxj = (valid && j > 0) ? ldg4(f.hx + c - nx) : zero;
        const float4 hzj = (valid && j > 0) ? ldg4(f.hz + c - nx) : zero;
        float hy_p = __shfl_up_sync(full, hy.w, 1);
        float hz_p = __shfl_up_sync(full, hz.w, 1);
        if (lane == 0) {
            hy_p = (valid && i0 > 0) ? __ldg(f.hy + c - 1) : 0.0f;
            hz_p = (valid && i0 > 0) ? __ldg(f.hz + c - 1) : 0.0f;
        }
        if (valid) {
            const float4 ex = ld4(f.ex + c), ey = ld4(f.ey + c), ez = ld4(f.ez + c);
            const uint32_t m4 = __ldg(reinterpret_cast<const uint32_t*>(f.mat + c));
            const bool any_gain = gain_on && (m4 & 0x80808080u);
            float4 jx = zero, jy = zero, jz = zero, n1 = zero, n2 = zero, n3 = zero;
            if (any_gain) {
                jx = ld4(f.jx + c); jy = ld4(f.jy + c); jz = ld4(f.jz + c);
                n1 = ld4(f.n1 + c); n2 = ld4(f.n2 + c); n3 = ld4(f.n3 + c);
            }
            float4 ex1, ey1, ez1;
            if (FACE && plane_has_flux(a.flux, true, w_xy, k))
                e_quad<true, true>(a, i0, j, k, c, hx, hy, hz, hxj, hzj, hxk, hyk, hy_p, hz_p, ex, ey,
                                   ez, m4, jx, jy, jz, n1, n2, n3, n, fl, ex1, ey1, ez1);
            else if (pml_xy || plane_in_z_slab(a, k))
                e_quad<false, true>(a, i0, j, k, c, hx, hy, hz, hxj, hzj, hxk, hyk, hy_p, hz_p, ex, ey,
                                    ez, m4, jx, jy, jz, n1, n2, n3, n, fl, ex1, ey1, ez1);
            else
                e_quad<false, false>(a, i0, j, k, c, hx, hy, hz, hxj, hzj, hxk, hyk, hy_p, hz_p, ex,
                                     ey, ez, m4, jx, jy, jz, n1, n2, n3, n, fl, ex1, ey1, ez1);
            st4(f.ex + c, ex1);
            st4(f.ey + c, ey1);
            st4(f.ez + c, ez1);
            if (any_gain) {
                st4(f.n1 + c, n1);
                st4(f.n2 + c, n2);
                st4(f.n3 + c, n3);
            }
        }
        hxk = hx;
        hyk = hy;
    }
}

__global__ void __launch_bounds__(256) k_e_vec(StepArgs a, int kz) {
    const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const bool valid = i0 < a.g.nx && j < a.g.ny;   // no early exit: shuffles and flux are warp-wide
    const long long n = a.step_ctr[0];
    const int k0 = blockIdx.z * kz;
    const int k1 = min(a.g.nz, k0 + kz);
    const int x0 = 4 * blockIdx.x * blockDim.x, xw = 4 * blockDim.x;
    const int y0 = blockIdx.y * blockDim.y;
    const bool face = tile_on_face(a.flux, x0, x0 + xw, y0, y0 + blockDim.y, k0, k1);
    const bool pml_xy = tile_in_xy_slab(a, x0, xw, y0, blockDim.y);
    if (face) {
        float fl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const bool w_xy = __any_sync(0xffffffffu, valid && cells_on_xy_face(a.flux, i0, 4, j));
        e_vec_walk<true>(a, i0, j, k0, k1, valid, pml_xy, n, fl, w_xy);
        flux_warp_reduce(a.flux, fl, warp_slot());
    } else {
        e_vec_walk<false>(a, i0, j, k0, k1, valid, pml_xy, n, nullptr, false);
    }
    finish_step(a);
}

bool vec_supported(const StepArgs& a) { return a.g.nx % 4 == 0; }

// ------------------------------------------------- TMA-staged E pass
// 2-D tile of BX x BY cells walking kz planes.  One thread streams each
// plane's H (with a -x / -y halo), E and material tiles into an S-slot
// shared-memory ring with bulk tensor copies (cp.async.bulk.tensor) that
// complete on per-slot mbarriers, S - 1 planes ahead of the compute.  The
// -z neighbour plane of Hx, Hy stays in registers; J and n of gain cells
// are loaded one plane ahead, once that plane's material tile has landed.
template <int BX, int BY, int S>
__global__ void __launch_bounds__(BX * BY) k_e_tma(StepArgs a, const __grid_constant__ TmaMaps maps,
                                                   int kz) {
    using Lay = TmaLayoutE<BX, BY>;
    constexpr int NW = BX * BY / 32;
    extern __shared__ unsigned char smem_raw[];
    __shared__ float wfl[6][NW];   // per-warp face-flux partials, summed plane by plane
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float* gbuf = reinterpret_cast<float*>(smem + S * Lay::kStage);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S * Lay::kStage + Lay::kGBytes);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int warp = tid >> 5;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
    const int i = x0 + tx, j = y0 + ty;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const uint32_t nxy = a.g.nxy;
    const bool valid = i < nx && j < ny;
    const int k0 = blockIdx.z * kz, k1 = min(nz, k0 + kz);
    const long long n = a.step_ctr[0];
    const bool face = tile_on_face(a.flux, x0, x0 + BX, y0, y0 + BY, k0, k1);
    const bool pml_xy = tile_in_xy_slab(a, x0, BX, y0, BY);
    // warp-uniform: the warp holds cells of an x or y face / of an x or y slab
    const bool w_xy = __any_sync(0xffffffffu, face && valid && cells_on_xy_face(a.flux, i, 1, j));
    const bool w_pml = __any_sync(0xffffffffu, pml_xy && valid && cell_in_xy_slab(a, i, j));
    const bool gain_on = a.gain.on;
    const DevFields& f = a.f;

    auto issue = [&](int s, int k) {
        unsigned char* p = smem + s * Lay::kStage;
        mbar_arrive_expect_tx(&bar[s], Lay::kTx);
        tma_load_3d(p + 0 * Lay::kHBytes, &maps.hx, x0 - 4, y0 - 1, k, &bar[s]);
        tma_load_3d(p + 1 * Lay::kHBytes, &maps.hy, x0 - 4, y0 - 1, k, &bar[s]);
        tma_load_3d(p + 2 * Lay::kHBytes, &maps.hz, x0 - 4, y0 - 1, k, &bar[s]);
        unsigned char* q = p + 3 * Lay::kHBytes;
        tma_load_3d(q + 0 * Lay::kEBytes, &maps.ex, x0, y0, k, &bar[s]);
        tma_load_3d(q + 1 * Lay::kEBytes, &maps.ey, x0, y0, k, &bar[s]);
        tma_load_3d(q + 2 * Lay::kEBytes, &maps.ez, x0, y0, k, &bar[s]);
        tma_load_3d(q + 3 * Lay::kEBytes, &maps.mat, x0, y0, k, &bar[s]);
    };
    auto mat_of = [&](int s) -> uint8_t {
        return (smem + s * Lay::kStage + 3 * Lay::kHBytes + 3 * Lay::kEBytes)[tid];
    };
    // J and n1..n3 of a gain cell, one plane ahead, into buffer b (no registers held)
    auto gslot = [&](int b, int q) -> float* { return gbuf + (b * 6 + q) * (BX * BY) + tid; };
    auto prefetch_gain = [&](int b, uint32_t cc) {
        cp_async_4(gslot(b, 0), f.jx + cc);
        cp_async_4(gslot(b, 1), f.jy + cc);
        cp_async_4(gslot(b, 2), f.jz + cc);
        cp_async_4(gslot(b, 3), f.n1 + cc);
        cp_async_4(gslot(b, 4), f.n2 + cc);
        cp_async_4(gslot(b, 5), f.n3 + cc);
    };

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        fence_barrier_init();
    }
    if (tid < 6 * NW) wfl[tid / NW][tid % NW] = 0.0f;
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < S && k0 + s < k1; ++s) issue(s, k0 + s);
    int issued = min(S, k1 - k0);   // planes issued into the ring so far
    bool block_fail = false;

    uint32_t c = valid ? (uint32_t)i + (uint32_t)nx * j + nxy * k0 : 0u;
    float hx_km1 = 0.0f, hy_km1 = 0.0f;
    if (valid && k0 > 0) {
        hx_km1 = __ldg(f.hx + c - nxy);
        hy_km1 = __ldg(f.hy + c - nxy);
    }
    bool fail = !mbar_wait_bounded(&bar[0], 0, kWaitLimit);
    bool pg = valid && gain_on && (mat_of(0) & 0x80);
    if (pg) prefetch_gain(0, c);
    cp_async_commit();
    for (int it = 0, k = k0; k < k1; ++it, ++k) {
        const int s = it % S;
        cp_async_wait_all();   // this plane's gain values (own thread's copies)
        bool ng = false;
        if (k + 1 < k1) {
            const int s1 = (it + 1) % S;
            fail |= !mbar_wait_bounded(&bar[s1], ((it + 1) / S) & 1, kWaitLimit);
            ng = valid && gain_on && (mat_of(s1) & 0x80);
            if (ng) prefetch_gain((it + 1) & 1, c + nxy);
        }
        cp_async_commit();
        float fl[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const bool fk = plane_has_flux(a.flux, face, w_xy, k);
        if (valid && !fail) {
            const unsigned char* p = smem + s * Lay::kStage;
            const float* Hx = reinterpret_cast<const float*>(p);
            const float* Hy = reinterpret_cast<const float*>(p + Lay::kHBytes);
            const float* Hz = reinterpret_cast<const float*>(p + 2 * Lay::kHBytes);
            const float* Ex = reinterpret_cast<const float*>(p + 3 * Lay::kHBytes);
            const float* Ey = reinterpret_cast<const float*>(p + 3 * Lay::kHBytes + Lay::kEBytes);
            const float* Ez = reinterpret_cast<const float*>(p + 3 * Lay::kHBytes + 2 * Lay::kEBytes);
            const int hc = (ty + 1) * (BX + 4) + tx + 4;
            HNb h;
            h.hx = Hx[hc];
            h.hy = Hy[hc];
            h.hz = Hz[hc];
            h.hy_i = Hy[hc - 1];
            h.hz_i = Hz[hc - 1];
            h.hx_j = Hx[hc - (BX + 4)];
            h.hz_j = Hz[hc - (BX + 4)];
            h.hx_k = hx_km1;
            h.hy_k = hy_km1;
            const uint8_t m = mat_of(s);
            const int b = it & 1;
            float jx = 0.f, jy = 0.f, jz = 0.f, n1 = 0.f, n2 = 0.f, n3 = 0.f;
            if (pg) {
                jx = *gslot(b, 0);
                jy = *gslot(b, 1);
                jz = *gslot(b, 2);
                n1 = *gslot(b, 3);
                n2 = *gslot(b, 4);
                n3 = *gslot(b, 5);
            }
            if (fk)
                e_apply<true, true>(a, i, j, k, c, h, m, Ex[tid], Ey[tid], Ez[tid], pg, jx, jy, jz, n1,
                                    n2, n3, n, fl);
            else if (w_pml || plane_in_z_slab(a, k))
                e_apply<false, true>(a, i, j, k, c, h, m, Ex[tid], Ey[tid], Ez[tid], pg, jx, jy, jz, n1,
                                     n2, n3, n, fl);
            else
                e_apply<false, false>(a, i, j, k, c, h, m, Ex[tid], Ey[tid], Ez[tid], pg, jx, jy, jz,
                                      n1, n2, n3, n, fl);
            hx_km1 = h.hx;
            hy_km1 = h.hy;
        }
        if (fk) {
            // this plane's flux terms: warp sums, added to the warp's partials
            const unsigned full = 0xffffffffu;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                float v = fl[q];
                if (__any_sync(full, v != 0.0f)) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
                    if ((tid & 31) == 0) wfl[q][warp] += v;
                }
            }
        }
        // slot s is free again; the barrier also ORs the threads' wait
        // verdicts, so every thread sees the same block_fail
        block_fail = __syncthreads_or(fail);
        if (block_fail) break;   // issue nothing more; drained below
        if (k + S < k1) {
            if (tid == 0) issue(s, k + S);
            issued = it + S + 1;
        }
        pg = ng;
        c += nxy;
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
            if (wfl[q][warp] != 0.0f) atomicAdd(a.flux.acc + q * kFluxSlots + (slot % kFluxSlots), (double)wfl[q][warp]);
    }
    finish_step(a);
}

// ------------------------------------------------------- TMA-staged H pass
// One thread per (i, j) walks the tile's planes; one thread streams the
// planes k0 .. k1 of E (with the +x/+y halo) and k0 .. k1-1 of H into an
// S-slot shared-memory ring with cp.async.bulk.tensor completing on
// mbarriers.  Plane p needs E of planes p and p+1, so iteration p waits for
// slot p+1 and frees slot p.  E beyond the grid is the TMA zero fill.  Gain
// blocks of the same launch run the Lorentz step as in the other variants.
template <int BX, int BY, int S>
__global__ void __launch_bounds__(BX * BY) k_hg_tma(StepArgs a, const __grid_constant__ TmaMaps maps,
                                                    HGLayout lay, int kz) {
    const long long n = a.step_ctr[0];
    unsigned idx;
    if (hg_block_kind(lay, blockIdx.x, idx)) {
        gain_block(a, idx, lay.q, n);
        return;
    }
    using Lay = TmaLayoutH<BX, BY>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S * Lay::kStage);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + BX * ty;
    const int bx = idx % lay.gx, by = (idx / lay.gx) % lay.gy, bz = idx / (lay.gx * lay.gy);
    const int x0 = bx * BX, y0 = by * BY;
    const int i = x0 + tx, j = y0 + ty;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const uint32_t nxy = a.g.nxy;
    const bool valid = i < nx && j < ny;
    const int k0 = bz * kz, k1 = min(nz, k0 + kz);
    const int planes = k1 - k0, total = planes + 1;
    const bool pml_xy = tile_in_xy_slab(a, x0, BX, y0, BY);
    const DevFields& f = a.f;

    auto issue = [&](int s, int p) {
        unsigned char* q = smem + s * Lay::kStage;
        const int k = k0 + p;
        mbar_arrive_expect_tx(&bar[s], p < planes ? Lay::kTx : Lay::kTxE);
        tma_load_3d(q + 0 * Lay::kEBytes, &maps.ebx, x0, y0, k, &bar[s]);
        tma_load_3d(q + 1 * Lay::kEBytes, &maps.eby, x0, y0, k, &bar[s]);
        tma_load_3d(q + 2 * Lay::kEBytes, &maps.ebz, x0, y0, k, &bar[s]);
        if (p < planes) {
            unsigned char* h = q + 3 * Lay::kEBytes;
            tma_load_3d(h + 0 * Lay::kHBytes, &maps.hsx, x0, y0, k, &bar[s]);
            tma_load_3d(h + 1 * Lay::kHBytes, &maps.hsy, x0, y0, k, &bar[s]);
            tma_load_3d(h + 2 * Lay::kHBytes, &maps.hsz, x0, y0, k, &bar[s]);
        }
    };

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < S && s < total; ++s) issue(s, s);
    int issued = min(S, total);   // planes issued into the ring so far
    bool block_fail = false;

    uint32_t c = valid ? (uint32_t)i + (uint32_t)nx * j + nxy * k0 : 0u;
    bool fail = !mbar_wait_bounded(&bar[0], 0, kWaitLimit);
    const int own = ty * (BX + 4) + tx;
    for (int p = 0; p < planes; ++p) {
        const int s = p % S, s1 = (p + 1) % S;
        const int k = k0 + p;
        fail |= !mbar_wait_bounded(&bar[s1], ((p + 1) / S) & 1, kWaitLimit);
        if (valid && !fail) {
            const float* E0 = reinterpret_cast<const float*>(smem + s * Lay::kStage);
            const float* E1 = reinterpret_cast<const float*>(smem + s1 * Lay::kStage);
            const float* Hs = reinterpret_cast<const float*>(smem + s * Lay::kStage + 3 * Lay::kEBytes);
            constexpr int EW = Lay::kEBytes / 4, HW = Lay::kHBytes / 4;
            ENb e;
            e.ex = E0[own];
            e.ey = E0[EW + own];
            e.ez = E0[2 * EW + own];
            e.ex_j1 = E0[own + BX + 4];
            e.ez_j1 = E0[2 * EW + own + BX + 4];
            e.ey_i1 = E0[EW + own + 1];
            e.ez_i1 = E0[2 * EW + own + 1];
            e.ex_k1 = E1[own];
            e.ey_k1 = E1[EW + own];
            float hx = Hs[tid], hy = Hs[HW + tid], hz = Hs[2 * HW + tid];
            if (pml_xy || plane_in_z_slab(a, k)) h_compute<true>(a, i, j, k, e, hx, hy, hz);
            else h_compute<false>(a, i, j, k, e, hx, hy, hz);
            f.hx[c] = hx;
            f.hy[c] = hy;
            f.hz[c] = hz;
        }
        // slot s is free again; the barrier also ORs the threads' wait
        // verdicts, so every thread sees the same block_fail
        block_fail = __syncthreads_or(fail);
        if (block_fail) break;   // issue nothing more; drained below
        if (p + S < total) {
            if (tid == 0) issue(s, p + S);
            issued = p + S + 1;
        }
        c += nxy;
    }
    if (block_fail) {
        // A wait gave up: record it, then give the copies still in flight a
        // bounded chance to land before the block's shared memory is released.
        if (tid == 0) atomicOr(a.err, 1);
        drain_ring(bar, S, issued, kWaitLimit);
    }
}

// -------------------------------------------------------------- launchers

HGLayout hg_layout(const StepArgs& a, const PassTune& t) {
    HGLayout L;
    const int cells_x = t.block.x * (t.variant == kVariantVec ? 4 : 1);
    L.gx = (a.g.nx + cells_x - 1) / cells_x;
    L.gy = (a.g.ny + t.block.y - 1) / t.block.y;
    const int zdiv = t.variant == kVariant3D ? (int)t.block.z : t.kz;
    L.gz = (a.g.nz + zdiv - 1) / zdiv;
    L.nH = L.gx * L.gy * L.gz;
    const int threads = t.block.x * t.block.y * (t.variant == kVariant3D ? t.block.z : 1);
    L.q = threads * kGainPerThread;
    L.nG = (a.gain.on && a.glist.count) ? (int)((a.glist.count + L.q - 1) / L.q) : 0;
    return L;
}

template <int BX, int BY>
static void launch_h_tma(const StepArgs& a, const HGLayout& L, int kz, const TmaMaps& maps,
                         cudaStream_t s) {
    const int smem = TmaLayoutH<BX, BY>::smem_bytes(kTmaStages);
    static bool attr_set = false;   // per instantiation, once per process
    if (!attr_set) {
        cudaFuncSetAttribute(k_hg_tma<BX, BY, kTmaStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
        attr_set = true;
    }
    k_hg_tma<BX, BY, kTmaStages><<<(unsigned)(L.nH + L.nG), dim3(BX, BY, 1), smem, s>>>(a, maps, L, kz);
}

void launch_h_pass(const StepArgs& a, const PassTune& t, const TmaMaps* tma, cudaStream_t s) {
    const HGLayout L = hg_layout(a, t);
    const unsigned blocks = (unsigned)(L.nH + L.nG);
    if (t.variant == kVariantTma && tma) {
        const int bx = t.block.x, by = t.block.y;
        if (bx == 32 && by == 4) return launch_h_tma<32, 4>(a, L, t.kz, *tma, s);
        if (bx == 32 && by == 8) return launch_h_tma<32, 8>(a, L, t.kz, *tma, s);
        if (bx == 64 && by == 4) return launch_h_tma<64, 4>(a, L, t.kz, *tma, s);
        if (bx == 64 && by == 8) return launch_h_tma<64, 8>(a, L, t.kz, *tma, s);
        if (bx == 128 && by == 2) return launch_h_tma<128, 2>(a, L, t.kz, *tma, s);
        if (bx == 128 && by == 4) return launch_h_tma<128, 4>(a, L, t.kz, *tma, s);
    }
    if (t.variant == kVariantVec && vec_supported(a)) {
        k_hg_vec<<<blocks, dim3(t.block.x, t.block.y, 1), 0, s>>>(a, L, t.kz);
    } else if (t.variant != kVariant3D) {
        k_hg_zmarch<<<blocks, dim3(t.block.x, t.block.y, 1), 0, s>>>(a, L, t.kz);
    } else {
        k_hg_3d<<<blocks, t.block, 0, s>>>(a, L);
    }
}

template <int BX, int BY>
static void launch_e_tma(const StepArgs& a, const PassTune& t, const TmaMaps& maps, cudaStream_t s) {
    const int smem = TmaLayoutE<BX, BY>::smem_bytes(kTmaStages);
    static bool attr_set = false;   // per instantiation, once per process
    if (!attr_set) {
        cudaFuncSetAttribute(k_e_tma<BX, BY, kTmaStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem);
        attr_set = true;
    }
    dim3 grid((a.g.nx + BX - 1) / BX, (a.g.ny + BY - 1) / BY, (a.g.nz + t.kz - 1) / t.kz);
    k_e_tma<BX, BY, kTmaStages><<<grid, dim3(BX, BY, 1), smem, s>>>(a, maps, t.kz);
}

bool tma_e_supported(const StepArgs& a) {
    // 16-byte global strides for the float and the uint8 maps
    return a.g.nx % 16 == 0;
}

// The CUDA driver API's tensor-map encoder, found through the runtime (no libcuda link).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool encode_box(CUtensorMap* m, CUtensorMapDataType dt, const void* base, int esize,
                const DevGrid& g, int bw, int bh) {
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * esize, (cuuint64_t)g.nx * g.ny * esize};
    const cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_tma(const StepArgs& a, int bx, int by, TmaMaps* out) {
    if (!tma_e_supported(a)) return false;
    const DevFields& f = a.f;
    const CUtensorMapDataType F32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    bool ok = encode_box(&out->ebx, F32, f.ex, 4, a.g, bx + 4, by + 1) &&
              encode_box(&out->eby, F32, f.ey, 4, a.g, bx + 4, by + 1) &&
              encode_box(&out->ebz, F32, f.ez, 4, a.g, bx + 4, by + 1) &&
              encode_box(&out->hsx, F32, f.hx, 4, a.g, bx, by) &&
              encode_box(&out->hsy, F32, f.hy, 4, a.g, bx, by) &&
              encode_box(&out->hsz, F32, f.hz, 4, a.g, bx, by) &&
              encode_box(&out->hx, F32, f.hx, 4, a.g, bx + 4, by + 1) &&
              encode_box(&out->hy, F32, f.hy, 4, a.g, bx + 4, by + 1) &&
              encode_box(&out->hz, F32, f.hz, 4, a.g, bx + 4, by + 1) &&
              encode_box(&out->ex, F32, f.ex, 4, a.g, bx, by) &&
              encode_box(&out->ey, F32, f.ey, 4, a.g, bx, by) &&
              encode_box(&out->ez, F32, f.ez, 4, a.g, bx, by) &&
              encode_box(&out->mat, CU_TENSOR_MAP_DATA_TYPE_UINT8, f.mat, 1, a.g, bx, by);
    return ok;
}

void launch_e_pass(const StepArgs& a, const PassTune& t, const TmaMaps* tma, cudaStream_t s) {
    if (t.variant == kVariantTma && tma) {
        const int bx = t.block.x, by = t.block.y;
        if (bx == 32 && by == 4) return launch_e_tma<32, 4>(a, t, *tma, s);
        if (bx == 32 && by == 8) return launch_e_tma<32, 8>(a, t, *tma, s);
        if (bx == 64 && by == 4) return launch_e_tma<64, 4>(a, t, *tma, s);
        if (bx == 64 && by == 8) return launch_e_tma<64, 8>(a, t, *tma, s);
        if (bx == 128 && by == 2) return launch_e_tma<128, 2>(a, t, *tma, s);
        if (bx == 128 && by == 4) return launch_e_tma<128, 4>(a, t, *tma, s);
    }
    if (t.variant == kVariantVec && vec_supported(a)) {
        dim3 grid((a.g.nx + 4 * t.block.x - 1) / (4 * t.block.x), (a.g.ny + t.block.y - 1) / t.block.y,
                  (a.g.nz + t.kz - 1) / t.kz);
        k_e_vec<<<grid, dim3(t.block.x, t.block.y, 1), 0, s>>>(a, t.kz);
    } else if (t.variant != kVariant3D) {
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
