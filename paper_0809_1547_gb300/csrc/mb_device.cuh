// Device-side data of one Maxwell–Bloch FDTD realization and the arithmetic
// of the two field passes.  Every kernel that advances a realization (the
// plain step in all its launch variants, the batched ensemble, the adjoint's
// forward recomputation) composes the same helpers below, so their results
// agree bit for bit.  The library is compiled with -fmad=false: every fused
// multiply-add is an explicit fmaf, so no kernel's inlining context can
// change the rounding.
//
// Units on the device are scaled so that FP32 stays far from under/overflow:
//   E_s = E/E0, H_s = eta0 H/E0, P_s = P/(eps0 E0), J_s = J dt/(eps0 E0),
//   n_i = N_i/N_a (i = 1..3; N0 = N_a (1 - n1 - n2 - n3) is not stored),
//   psi_E,s = psi_E eta0 dx/E0, psi_H,s = psi_H dx/E0,
// with E0 = sqrt(hbar w0 n_ref / eps0).  In these units the Yee step reads
//   H_s -= S (dE_s + psi_H,s),          S = c dt/dx,
//   E_s += (1/eps_r) (S (dH_s + psi_E,s) - J_s - J_src,s).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mb {

// Cell offsets are 32-bit: a realization holds fewer than 2^32 cells.
struct DevGrid {
    int nx, ny, nz;
    uint32_t nxy, ncell;
};

// The face flux is accumulated into kFluxSlots FP64 slots per face (spread
// over L2 to avoid serialising the atomics); read-outs sum the slots.
constexpr int kFluxSlots = 64;

struct DevFields {
    float *ex, *ey, *ez, *hx, *hy, *hz;
    float *px, *py, *pz, *jx, *jy, *jz;
    float *n1, *n2, *n3;
    const uint8_t* mat;        // bits 0..6: material id, bit 7: gain medium
    const float* inv_eps;      // dense 1/eps_r per cell, or nullptr
    const float* lut_inv_eps;  // 1/eps_r per material id (128 entries)
    // a map of at most two eps_r values (n_lut <= 2): 1/eps_r of ids 0 and 1
    // (the table's first entries), chosen by a select instead of a load
    int n_lut;
    float ie0, ie1;
};

// CPML memories live only in the slabs: for axis w, 2 L layers indexed by
// s = i (i < L) or s = i - n + 2L (i >= n - L).  Four planes per slab axis:
// f = 0, 1: the two E components with a w-derivative, f = 2, 3: the two H
// components.  x-slab index ((f nz + k) ny + j) 2L + s, y-slab
// ((f nz + k) 2L + s) nx + i, z-slab ((f zn + s) ny + j) nx + i.
// Along z the slab region is stated by its bounds: plane k lies in it when
// k < zlo or k >= zhi, at layer s = k (k < zlo) or s = k - zhi + zs, with zn
// layers stored.  A whole grid has zlo = L, zhi = nz - L, zs = L, zn = 2L
// (the same layers as x and y); a z-slab of a grid split along z holds only
// the CPML planes of the whole grid that fall inside it.
struct DevCpml {
    int L;
    int zlo, zhi, zs, zn;
    float *psx, *psy, *psz;
    const float *bex, *cex, *bhx, *chx;
    const float *bey, *cey, *bhy, *chy;
    const float *bez, *cez, *bhz, *chz;
};

// Gain medium, scaled: J_s' = cJ1 J_s + cJE (n1 - n2) E_s - cJP P_s
//                            + cJN sqrt(max(n2,0) + nfloor) zeta,
// n_i' = n_i + g_i + sum_j G_ij n_j + mk_i S_pop, S_pop = (E_s + E_s').J_s'/2.
struct DevGain {
    int on;
    float cJ1, cJE, cJP, cJN, nfloor;
    float g[3];
    float G[3][3];
    float mk[3];
    uint32_t key0, key1;
    // index of the realization's cell that local cell 0 is: the noise is
    // keyed by the cell's index in the whole grid (0 unless this is a
    // z-slab of a grid split along z)
    uint32_t cell0;
};

// Soft current source: the scaled current of step n is wave[n - n0] for
// n0 <= n < n0 + count and zero elsewhere (tabulated on the host in FP64 over
// the window where the Gaussian envelope is above ~1e-60).
struct DevSource {
    int on, comp;
    int64_t cell;
    long long n0;
    int count;
    const float* wave;
};

// Outward Poynting flux of the interior box [r0, r1) per axis through the
// planes plo / phi, accumulated in FP64 (scaled units).
struct DevFlux {
    int on;
    int plo[3], phi[3];
    int r0[3], r1[3];
    double* acc;   // [6][kFluxSlots]: faces x-, x+, y-, y+, z-, z+
};

// Gain cells in increasing cell order (static for a material): the Lorentz
// update runs over this list so that whole warps do gain work.
struct DevGainList {
    const uint32_t* cell;
    uint32_t count;
};

struct StepArgs {
    DevGrid g;
    DevFields f;
    DevCpml pml;
    DevGain gain;
    DevGainList glist;
    DevSource src;
    DevFlux flux;
    float S;
    // [0]: steps completed so far = index n of the step in progress; the
    // last block of the E pass increments it.  [1]: blocks of the current E
    // pass that have finished (reset to 0 by the last one).
    long long* step_ctr;
    // Set (bit 0) when a bounded device wait gave up; read by the host.
    int* err;
};

// Where a cell update writes the CPML memories it advances: the step's own
// arrays (in-place passes) or the other copy of them (single-pass step).
struct PsiOut {
    float *x, *y, *z;
};

__device__ __forceinline__ PsiOut psi_in_place(const StepArgs& a) {
    return PsiOut{a.pml.psx, a.pml.psy, a.pml.psz};
}

// Destination of the single-pass step: E^{n+1}, H^{n+1/2} and the advanced
// CPML memories go to a second copy of those arrays (the source copy is
// read-only during the launch, so tiles can recompute their neighbours'
// edge H values from it); P, J and the populations stay in place.
struct DevPing {
    float *ex, *ey, *ez, *hx, *hy, *hz;
    PsiOut psi;
    // the step count after this step is also stored here, for the probes of
    // the copy the step writes (they may run during the next step, which
    // advances the main counter)
    long long* sample;
};

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies mixing the counter with a key bumped by two Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// u = ((x >> 9) + 1/2) 2^-23: exact in FP32, strictly inside (0, 1).  Formed
// as (1 + (x >> 9) 2^-23) - (1 - 2^-24), the first term by placing the 23
// bits under the exponent of 1; both terms lie in [1/2, 2], so the
// difference is exact (Sterbenz).
__device__ __forceinline__ float u32_to_unit(uint32_t x) {
    return __uint_as_float((x >> 9) | 0x3F800000u) - 0.99999994039535522f;
}

// Three standard normals of cell `cell` at step `step`: Box–Muller,
// z0 + i z1 = sqrt(-2 ln u0) exp(2 pi i u1), z2 = sqrt(-2 ln u2) cos(2 pi u3).
// FP32 on the special-function unit: ln via __logf (absolute error below
// 2^-21 on [0.5, 2], 3 ulp elsewhere), sqrt(q) as q rsqrt(q) (q > 0 since
// u < 1), and the angle taken as 2 pi (u - 1/2) in [-pi, pi), where __sincosf
// is accurate to 2^-21 absolute: cos(2 pi u) = -cos(2 pi (u - 1/2)), likewise
// for sin.  The resulting normals differ from exact ones by ~1e-7 in rms.
__device__ __forceinline__ void langevin_normals(uint32_t cell, uint32_t step, uint32_t k0,
                                                 uint32_t k1, float& z0, float& z1, float& z2) {
    const uint4 x = philox4x32_10(make_uint4(cell, step, 0u, 0u), k0, k1);
    const float u0 = u32_to_unit(x.x), u1 = u32_to_unit(x.y);
    const float u2 = u32_to_unit(x.z), u3 = u32_to_unit(x.w);
    const float q01 = -2.0f * __logf(u0);
    const float q23 = -2.0f * __logf(u2);
    const float r01 = q01 * rsqrtf(q01);
    const float r23 = q23 * rsqrtf(q23);
    const float two_pi = 6.283185307179586f;
    float s1, c1;
    __sincosf(two_pi * (u1 - 0.5f), &s1, &c1);
    const float c3 = __cosf(two_pi * (u3 - 0.5f));
    z0 = -r01 * c1;
    z1 = -r01 * s1;
    z2 = -r23 * c3;
}

__device__ __forceinline__ int slab_index(int i, int n, int L) {
    return (i < L) ? i : i - n + 2 * L;
}

// E values the H update of one cell reads: its own three components and the
// +x / +y / +z neighbours that enter the forward differences.
struct ENb {
    float ex, ey, ez, ex_j1, ex_k1, ey_i1, ey_k1, ez_i1, ez_j1;
};

// H values the E update of one cell reads: its own three components and the
// -x / -y / -z neighbours that enter the backward differences.
struct HNb {
    float hx, hy, hz, hx_j, hx_k, hy_i, hy_k, hz_i, hz_j;
};

// Neighbours from global memory (E is read-only during the H pass); fields
// beyond the last cell are zero.
__device__ __forceinline__ ENb load_e_nbrs(const StepArgs& a, int i, int j, int k, uint32_t c) {
    const DevFields& f = a.f;
    const int nx = a.g.nx;
    const uint32_t nxy = a.g.nxy;
    ENb e;
    e.ex = __ldg(f.ex + c);
    e.ey = __ldg(f.ey + c);
    e.ez = __ldg(f.ez + c);
    const bool xi = i + 1 < nx, yj = j + 1 < a.g.ny, zk = k + 1 < a.g.nz;
    e.ex_j1 = yj ? __ldg(f.ex + c + nx) : 0.0f;
    e.ex_k1 = zk ? __ldg(f.ex + c + nxy) : 0.0f;
    e.ey_i1 = xi ? __ldg(f.ey + c + 1) : 0.0f;
    e.ey_k1 = zk ? __ldg(f.ey + c + nxy) : 0.0f;
    e.ez_i1 = xi ? __ldg(f.ez + c + 1) : 0.0f;
    e.ez_j1 = yj ? __ldg(f.ez + c + nx) : 0.0f;
    return e;
}

// H is read-only during the E pass; fields before the first cell are zero.
__device__ __forceinline__ HNb load_h_nbrs(const StepArgs& a, int i, int j, int k, uint32_t c) {
    const DevFields& f = a.f;
    const int nx = a.g.nx;
    const uint32_t nxy = a.g.nxy;
    HNb h;
    h.hx = __ldg(f.hx + c);
    h.hy = __ldg(f.hy + c);
    h.hz = __ldg(f.hz + c);
    h.hx_j = (j > 0) ? __ldg(f.hx + c - nx) : 0.0f;
    h.hx_k = (k > 0) ? __ldg(f.hx + c - nxy) : 0.0f;
    h.hy_i = (i > 0) ? __ldg(f.hy + c - 1) : 0.0f;
    h.hy_k = (k > 0) ? __ldg(f.hy + c - nxy) : 0.0f;
    h.hz_i = (i > 0) ? __ldg(f.hz + c - 1) : 0.0f;
    h.hz_j = (j > 0) ? __ldg(f.hz + c - nx) : 0.0f;
    return h;
}

// ------------------------------------------------------------- H half-step
// CPML of the H update at cell (i, j, k): advances psi_H and adds it to the
// curl components.  d = (dEz_dy, dEy_dz, dEx_dz, dEz_dx, dEy_dx, dEx_dy).
// Reads the memories of the step's own arrays (a.pml) and, with WR, writes
// the advanced ones to o (the same arrays for an in-place step).
template <bool WR>
__device__ __forceinline__ void h_pml(const StepArgs& a, int i, int j, int k, const float d[6],
                                      float& cx, float& cy, float& cz, const PsiOut& o) {
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const int L = a.pml.L;
    const int L2 = 2 * L;
    if (i < L || i >= nx - L) {
        const uint32_t s = slab_index(i, nx, L);
        const uint32_t plane = (uint32_t)nz * ny * L2;
        const uint32_t q = ((uint32_t)k * ny + j) * L2 + s;
        const float b = __ldg(a.pml.bhx + i), cc = __ldg(a.pml.chx + i);
        const float* p = a.pml.psx;
        const float psi_yx = fmaf(b, p[q + 2 * plane], cc * d[3]);   // Hy: d/dx Ez
        const float psi_zx = fmaf(b, p[q + 3 * plane], cc * d[4]);   // Hz: d/dx Ey
        if (WR) {
            o.x[q + 2 * plane] = psi_yx;
            o.x[q + 3 * plane] = psi_zx;
        }
        cy -= psi_yx;
        cz += psi_zx;
    }
    if (j < L || j >= ny - L) {
        const uint32_t s = slab_index(j, ny, L);
        const uint32_t plane = (uint32_t)nz * L2 * nx;
        const uint32_t q = ((uint32_t)k * L2 + s) * nx + i;
        const float b = __ldg(a.pml.bhy + j), cc = __ldg(a.pml.chy + j);
        const float* p = a.pml.psy;
        const float psi_xy = fmaf(b, p[q + 2 * plane], cc * d[0]);   // Hx: d/dy Ez
        const float psi_zy = fmaf(b, p[q + 3 * plane], cc * d[5]);   // Hz: d/dy Ex
        if (WR) {
            o.y[q + 2 * plane] = psi_xy;
            o.y[q + 3 * plane] = psi_zy;
        }
        cx += psi_xy;
        cz -= psi_zy;
    }
    if (k < a.pml.zlo || k >= a.pml.zhi) {
        const uint32_t s = (k < a.pml.zlo) ? k : k - a.pml.zhi + a.pml.zs;
        const uint32_t plane = (uint32_t)a.pml.zn * ny * nx;
        const uint32_t q = (s * ny + j) * nx + i;
        const float b = __ldg(a.pml.bhz + k), cc = __ldg(a.pml.chz + k);
        const float* p = a.pml.psz;
        const float psi_xz = fmaf(b, p[q + 2 * plane], cc * d[1]);   // Hx: d/dz Ey
        const float psi_yz = fmaf(b, p[q + 3 * plane], cc * d[2]);   // Hy: d/dz Ex
        if (WR) {
            o.z[q + 2 * plane] = psi_xz;
            o.z[q + 3 * plane] = psi_yz;
        }
        cx -= psi_xz;
        cy += psi_yz;
    }
}

// Prefetch into L1 the lines of the CPML memories that the update of cell
// (i, j, k) will read (the E memories, planes 0 and 1 of each slab array,
// or the H memories, planes 2 and 3), so a later load finds them on chip.
__device__ __forceinline__ void prefetch_l1(const float* p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}
__device__ __forceinline__ void prefetch_psi(const StepArgs& a, int i, int j, int k, int f0) {
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const int L = a.pml.L;
    const int L2 = 2 * L;
    if (i < L || i >= nx - L) {
        const uint32_t plane = (uint32_t)nz * ny * L2;
        const uint32_t q = ((uint32_t)k * ny + j) * L2 + slab_index(i, nx, L);
        prefetch_l1(a.pml.psx + q + f0 * plane);
        prefetch_l1(a.pml.psx + q + (f0 + 1) * plane);
    }
    if (j < L || j >= ny - L) {
        const uint32_t plane = (uint32_t)nz * L2 * nx;
        const uint32_t q = ((uint32_t)k * L2 + slab_index(j, ny, L)) * nx + i;
        prefetch_l1(a.pml.psy + q + f0 * plane);
        prefetch_l1(a.pml.psy + q + (f0 + 1) * plane);
    }
    if (k < a.pml.zlo || k >= a.pml.zhi) {
        const uint32_t s = (k < a.pml.zlo) ? k : k - a.pml.zhi + a.pml.zs;
        const uint32_t plane = (uint32_t)a.pml.zn * ny * nx;
        const uint32_t q = (s * ny + j) * nx + i;
        prefetch_l1(a.pml.psz + q + f0 * plane);
        prefetch_l1(a.pml.psz + q + (f0 + 1) * plane);
    }
}

// H^{n+1/2} = H^{n-1/2} - S (curl_fwd E^n + psi_H) for cell (i, j, k), on
// H values held in registers.  PML: the cell may lie in a CPML slab (false
// only when it surely does not).  The advanced CPML memories go to o (WR).
template <bool PML, bool WR>
__device__ __forceinline__ void h_compute_to(const StepArgs& a, int i, int j, int k, const ENb& e,
                                             float& hx, float& hy, float& hz, const PsiOut& o) {
    float d[6];
    d[0] = e.ez_j1 - e.ez;   // dEz_dy
    d[1] = e.ey_k1 - e.ey;   // dEy_dz
    d[2] = e.ex_k1 - e.ex;   // dEx_dz
    d[3] = e.ez_i1 - e.ez;   // dEz_dx
    d[4] = e.ey_i1 - e.ey;   // dEy_dx
    d[5] = e.ex_j1 - e.ex;   // dEx_dy
    float cx = d[0] - d[1];
    float cy = d[2] - d[3];
    float cz = d[4] - d[5];
    if (PML && a.pml.L > 0) h_pml<WR>(a, i, j, k, d, cx, cy, cz, o);
    const float S = a.S;
    hx = fmaf(-S, cx, hx);
    hy = fmaf(-S, cy, hy);
    hz = fmaf(-S, cz, hz);
}

template <bool PML>
__device__ __forceinline__ void h_compute(const StepArgs& a, int i, int j, int k, const ENb& e,
                                          float& hx, float& hy, float& hz) {
    h_compute_to<PML, true>(a, i, j, k, e, hx, hy, hz, psi_in_place(a));
}

// The same update read from and written to global memory at cell c.
template <bool PML>
__device__ __forceinline__ void h_core(const StepArgs& a, int i, int j, int k, uint32_t c,
                                       const ENb& e) {
    const DevFields& f = a.f;
    float hx = f.hx[c], hy = f.hy[c], hz = f.hz[c];
    h_compute<PML>(a, i, j, k, e, hx, hy, hz);
    f.hx[c] = hx;
    f.hy[c] = hy;
    f.hz[c] = hz;
}

__device__ __forceinline__ void h_update_cell(const StepArgs& a, int i, int j, int k) {
    const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
    h_core<true>(a, i, j, k, c, load_e_nbrs(a, i, j, k, c));
}

// Soft current J_src,s at t = (n + 1/2) dt.
__device__ __forceinline__ float source_value(const DevSource& s, long long n) {
    const long long q = n - s.n0;
    return (q >= 0 && q < s.count) ? __ldg(s.wave + q) : 0.0f;
}

// --------------------------------------------- gain medium (gain cells only)
// Lorentz polarization with the Langevin force of step n:
// J^{n+1/2} (in j*) and P^{n+1} (in p*) from J^{n-1/2}, P^n, E^n, N^n.
__device__ __forceinline__ void lorentz_step(const DevGain& G, uint32_t c, long long n,
                                             float ex0, float ey0, float ez0, float n1, float n2,
                                             float& jx, float& jy, float& jz,
                                             float& px, float& py, float& pz) {
    const float dn = n1 - n2;
    const float amp = G.cJN * sqrtf(fmaxf(n2, 0.0f) + G.nfloor);
    float z0, z1, z2;
    langevin_normals(c + G.cell0, (uint32_t)n, G.key0, G.key1, z0, z1, z2);
    const float kE = G.cJE * dn;
    jx = fmaf(amp, z0, fmaf(-G.cJP, px, fmaf(kE, ex0, G.cJ1 * jx)));
    jy = fmaf(amp, z1, fmaf(-G.cJP, py, fmaf(kE, ey0, G.cJ1 * jy)));
    jz = fmaf(amp, z2, fmaf(-G.cJP, pz, fmaf(kE, ez0, G.cJ1 * jz)));
    px = px + jx;
    py = py + jy;
    pz = pz + jz;
}

// Crank–Nicolson populations driven by S_pop = (E^n + E^{n+1}) . J^{n+1/2} / 2.
__device__ __forceinline__ void population_step(const DevGain& G, float ex0, float ey0, float ez0,
                                                float ex1, float ey1, float ez1, float jx,
                                                float jy, float jz, float& n1, float& n2,
                                                float& n3) {
    const float sp =
        0.5f * fmaf(ez0 + ez1, jz, fmaf(ey0 + ey1, jy, (ex0 + ex1) * jx));
    float d[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        d[r] = fmaf(G.mk[r], sp, fmaf(G.G[r][2], n3, fmaf(G.G[r][1], n2, fmaf(G.G[r][0], n1, G.g[r]))));
    const float a1 = n1 + d[0];
    const float a2 = n2 + d[1];
    const float a3 = n3 + d[2];
    n1 = a1;
    n2 = a2;
    n3 = a3;
}

// --------------------------------------------------------------- E update
// CPML of the E update: advances psi_E and adds it to the curl components.
// d = (dHz_dy, dHy_dz, dHx_dz, dHz_dx, dHy_dx, dHx_dy).
__device__ __forceinline__ void e_pml(const StepArgs& a, int i, int j, int k, const float d[6],
                                      float& cx, float& cy, float& cz, const PsiOut& o) {
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
    const int L = a.pml.L;
    const int L2 = 2 * L;
    if (i < L || i >= nx - L) {
        const uint32_t s = slab_index(i, nx, L);
        const uint32_t plane = (uint32_t)nz * ny * L2;
        const uint32_t q = ((uint32_t)k * ny + j) * L2 + s;
        const float b = __ldg(a.pml.bex + i), cc = __ldg(a.pml.cex + i);
        const float* p = a.pml.psx;
        const float psi_yx = fmaf(b, p[q], cc * d[3]);            // Ey: d/dx Hz
        const float psi_zx = fmaf(b, p[q + plane], cc * d[4]);    // Ez: d/dx Hy
        o.x[q] = psi_yx;
        o.x[q + plane] = psi_zx;
        cy -= psi_yx;
        cz += psi_zx;
    }
    if (j < L || j >= ny - L) {
        const uint32_t s = slab_index(j, ny, L);
        const uint32_t plane = (uint32_t)nz * L2 * nx;
        const uint32_t q = ((uint32_t)k * L2 + s) * nx + i;
        const float b = __ldg(a.pml.bey + j), cc = __ldg(a.pml.cey + j);
        const float* p = a.pml.psy;
        const float psi_xy = fmaf(b, p[q], cc * d[0]);            // Ex: d/dy Hz
        const float psi_zy = fmaf(b, p[q + plane], cc * d[5]);    // Ez: d/dy Hx
        o.y[q] = psi_xy;
        o.y[q + plane] = psi_zy;
        cx += psi_xy;
        cz -= psi_zy;
    }
    if (k < a.pml.zlo || k >= a.pml.zhi) {
        const uint32_t s = (k < a.pml.zlo) ? k : k - a.pml.zhi + a.pml.zs;
        const uint32_t plane = (uint32_t)a.pml.zn * ny * nx;
        const uint32_t q = (s * ny + j) * nx + i;
        const float b = __ldg(a.pml.bez + k), cc = __ldg(a.pml.cez + k);
        const float* p = a.pml.psz;
        const float psi_xz = fmaf(b, p[q], cc * d[1]);            // Ex: d/dz Hy
        const float psi_yz = fmaf(b, p[q + plane], cc * d[2]);    // Ey: d/dz Hx
        o.z[q] = psi_xz;
        o.z[q + plane] = psi_yz;
        cx -= psi_xz;
        cy += psi_yz;
    }
}

// E^{n+1} from E^n, the backward curl of H^{n+1/2} (+ psi_E), the total
// current (Lorentz J^{n+1/2} plus source) and the PEC walls.
template <bool PML>
__device__ __forceinline__ void e_field_step(const StepArgs& a, int i, int j, int k, uint32_t c,
                                             const HNb& h, float ie, float ex0, float ey0,
                                             float ez0, float sx, float sy, float sz, long long n,
                                             float& ex1, float& ey1, float& ez1, const PsiOut& o) {
    float d[6];
    d[0] = h.hz - h.hz_j;   // dHz_dy
    d[1] = h.hy - h.hy_k;   // dHy_dz
    d[2] = h.hx - h.hx_k;   // dHx_dz
    d[3] = h.hz - h.hz_i;   // dHz_dx
    d[4] = h.hy - h.hy_i;   // dHy_dx
    d[5] = h.hx - h.hx_j;   // dHx_dy
    float cx = d[0] - d[1];
    float cy = d[2] - d[3];
    float cz = d[4] - d[5];
    if (PML && a.pml.L > 0) e_pml(a, i, j, k, d, cx, cy, cz, o);
    if (a.src.on && c == (uint32_t)a.src.cell) {
        const float v = source_value(a.src, n);
        if (a.src.comp == 0) sx += v;
        else if (a.src.comp == 1) sy += v;
        else sz += v;
    }
    const float S = a.S;
    ex1 = fmaf(ie, fmaf(S, cx, -sx), ex0);
    ey1 = fmaf(ie, fmaf(S, cy, -sy), ey0);
    ez1 = fmaf(ie, fmaf(S, cz, -sz), ez0);
    // PEC walls: tangential E on the planes i = 0, j = 0, k = 0.
    if (j == 0 || k == 0) ex1 = 0.0f;
    if (i == 0 || k == 0) ey1 = 0.0f;
    if (i == 0 || j == 0) ez1 = 0.0f;
}

// Outward face-flux terms of cell (i, j, k): (E^n + E^{n+1})/2 on the face
// plane against H^{n+1/2} half a cell below it, added into fl[6].
__device__ __forceinline__ void flux_terms(const DevFlux& F, int i, int j, int k, const HNb& h,
                                           float ex0, float ey0, float ez0, float ex1, float ey1,
                                           float ez1, float fl[6]) {
    const float mx = 0.5f * (ex0 + ex1), my = 0.5f * (ey0 + ey1), mz = 0.5f * (ez0 + ez1);
    if (j >= F.r0[1] && j < F.r1[1] && k >= F.r0[2] && k < F.r1[2]) {
        const float s = fmaf(my, h.hz_i, -(mz * h.hy_i));
        if (i == F.plo[0]) fl[0] -= s;
        if (i == F.phi[0]) fl[1] += s;
    }
    if (i >= F.r0[0] && i < F.r1[0] && k >= F.r0[2] && k < F.r1[2]) {
        const float s = fmaf(mz, h.hx_j, -(mx * h.hz_j));
        if (j == F.plo[1]) fl[2] -= s;
        if (j == F.phi[1]) fl[3] += s;
    }
    if (i >= F.r0[0] && i < F.r1[0] && j >= F.r0[1] && j < F.r1[1]) {
        const float s = fmaf(mx, h.hy_k, -(my * h.hx_k));
        if (k == F.plo[2]) fl[4] -= s;
        if (k == F.phi[2]) fl[5] += s;
    }
}

// ------------------------------------------------- Lorentz step, gain cells
// J^{n+1/2} and P^{n+1} of gain cell c with the Langevin force of step n.
// It reads only time-n state (E^n, P^n, J^{n-1/2}, N^n), so it runs in the
// H half-step launch, before the E pass overwrites E.
__device__ __forceinline__ void gain_cell_step(const StepArgs& a, uint32_t c, long long n) {
    const DevFields& f = a.f;
    const float ex0 = __ldg(f.ex + c), ey0 = __ldg(f.ey + c), ez0 = __ldg(f.ez + c);
    const float n1 = f.n1[c], n2 = f.n2[c];
    float px = f.px[c], py = f.py[c], pz = f.pz[c];
    float jx = f.jx[c], jy = f.jy[c], jz = f.jz[c];
    lorentz_step(a.gain, c, n, ex0, ey0, ez0, n1, n2, jx, jy, jz, px, py, pz);
    f.jx[c] = jx;
    f.jy[c] = jy;
    f.jz[c] = jz;
    f.px[c] = px;
    f.py[c] = py;
    f.pz[c] = pz;
}

// ------------------------------------------------ E / population pass
// One cell, after the gain cells' Lorentz step of this time step: E^{n+1}
// with the current J^{n+1/2}, then N^{n+1}; with FLUX, the face-flux terms.
// The E / population update of cell c from its loaded inputs: material byte
// m, E^n, and for gain cells J^{n+1/2} and n1..n3 at time n.
// In registers: E^{n+1} into ex1..ez1 and, for gain cells, N^{n+1} into
// n1..n3 (in place); face-flux terms into fl with FLUX.
// With 1/eps_r of the cell given (ie); the advanced CPML memories go to o.
template <bool FLUX, bool PML>
__device__ __forceinline__ void e_compute_ie(const StepArgs& a, int i, int j, int k, uint32_t c,
                                             const HNb& h, float ie, float ex0, float ey0,
                                             float ez0, bool gain, float jx, float jy, float jz,
                                             float& n1, float& n2, float& n3, long long n,
                                             float fl[6], float& ex1, float& ey1, float& ez1,
                                             const PsiOut& o, bool flux_plane = true) {
    e_field_step<PML>(a, i, j, k, c, h, ie, ex0, ey0, ez0, jx, jy, jz, n, ex1, ey1, ez1, o);
    if (gain) population_step(a.gain, ex0, ey0, ez0, ex1, ey1, ez1, jx, jy, jz, n1, n2, n3);
    if (FLUX && a.flux.on && flux_plane) flux_terms(a.flux, i, j, k, h, ex0, ey0, ez0, ex1, ey1, ez1, fl);
}

// The advanced CPML memories go to o.
template <bool FLUX, bool PML>
__device__ __forceinline__ void e_compute_to(const StepArgs& a, int i, int j, int k, uint32_t c,
                                             const HNb& h, uint8_t m, float ex0, float ey0,
                                             float ez0, bool gain, float jx, float jy, float jz,
                                             float& n1, float& n2, float& n3, long long n,
                                             float fl[6], float& ex1, float& ey1, float& ez1,
                                             const PsiOut& o, bool flux_plane = true) {
    const DevFields& f = a.f;
    const float ie = f.inv_eps       ? __ldg(f.inv_eps + c)
                     : f.n_lut <= 2 ? ((m & 0x7f) ? f.ie1 : f.ie0)
                                    : __ldg(f.lut_inv_eps + (m & 0x7f));
    e_compute_ie<FLUX, PML>(a, i, j, k, c, h, ie, ex0, ey0, ez0, gain, jx, jy, jz, n1, n2, n3, n,
                            fl, ex1, ey1, ez1, o, flux_plane);
}

template <bool FLUX, bool PML>
__device__ __forceinline__ void e_compute(const StepArgs& a, int i, int j, int k, uint32_t c,
                                          const HNb& h, uint8_t m, float ex0, float ey0, float ez0,
                                          bool gain, float jx, float jy, float jz, float& n1,
                                          float& n2, float& n3, long long n, float fl[6],
                                          float& ex1, float& ey1, float& ez1,
                                          bool flux_plane = true) {
    e_compute_to<FLUX, PML>(a, i, j, k, c, h, m, ex0, ey0, ez0, gain, jx, jy, jz, n1, n2, n3, n,
                            fl, ex1, ey1, ez1, psi_in_place(a), flux_plane);
}

template <bool FLUX, bool PML>
__device__ __forceinline__ void e_apply(const StepArgs& a, int i, int j, int k, uint32_t c,
                                        const HNb& h, uint8_t m, float ex0, float ey0, float ez0,
                                        bool gain, float jx, float jy, float jz, float n1, float n2,
                                        float n3, long long n, float fl[6], bool flux_plane = true) {
    const DevFields& f = a.f;
    float ex1, ey1, ez1;
    e_compute<FLUX, PML>(a, i, j, k, c, h, m, ex0, ey0, ez0, gain, jx, jy, jz, n1, n2, n3, n, fl,
                         ex1, ey1, ez1, flux_plane);
    f.ex[c] = ex1;
    f.ey[c] = ey1;
    f.ez[c] = ez1;
    if (gain) {
        f.n1[c] = n1;
        f.n2[c] = n2;
        f.n3[c] = n3;
    }
}

template <bool FLUX, bool PML>
__device__ __forceinline__ void e_core(const StepArgs& a, int i, int j, int k, uint32_t c,
                                       const HNb& h, long long n, float fl[6],
                                       bool flux_plane = true) {
    const DevFields& f = a.f;
    const uint8_t m = __ldg(f.mat + c);
    const bool gain = a.gain.on && (m & 0x80);
    const float ex0 = f.ex[c], ey0 = f.ey[c], ez0 = f.ez[c];
    float jx = 0.0f, jy = 0.0f, jz = 0.0f;
    float n1 = 0.0f, n2 = 0.0f, n3 = 0.0f;
    if (gain) {
        jx = f.jx[c];
        jy = f.jy[c];
        jz = f.jz[c];
        n1 = f.n1[c];
        n2 = f.n2[c];
        n3 = f.n3[c];
    }
    e_apply<FLUX, PML>(a, i, j, k, c, h, m, ex0, ey0, ez0, gain, jx, jy, jz, n1, n2, n3, n, fl,
                       flux_plane);
}

template <bool FLUX>
__device__ __forceinline__ void e_update_cell(const StepArgs& a, int i, int j, int k,
                                              long long n, float fl[6]) {
    const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
    e_core<FLUX, true>(a, i, j, k, c, load_h_nbrs(a, i, j, k, c), n, fl);
}

// Warp-level flux reduction: FP32 sums within the warp (skipped for faces
// no lane touches), one FP64 atomic per warp and face into a slot.  Every
// lane of the warp must call it.
__device__ __forceinline__ void flux_warp_reduce(const DevFlux& F, const float fl[6], unsigned slot) {
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        float v = fl[q];
        if (__any_sync(full, v != 0.0f)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(F.acc + q * kFluxSlots + (slot % kFluxSlots), (double)v);
        }
    }
}

}  // namespace mb
