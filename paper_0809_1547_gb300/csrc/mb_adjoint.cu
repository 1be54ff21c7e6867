// Reverse-time discrete adjoint of the Maxwell–Bloch step: the gradient of
// the energy crossing a z plane with respect to the per-cell permittivity
// and the pump rate, with forward checkpoints and per-segment recomputation.
//
// Forward step n (device units, gain terms in gain cells only):
//   H'  = H - S (curl_f E + psi_H),            psi_H' = b_H psi_H + c_H dE
//   J'  = cJ1 J + cJE (n1 - n2) E - cJP P + amp(n2) zeta,   P' = P + J'
//   E'  = mask (E + ie (S (curl_b H' + psi_E) - J' - src)),  psi_E' = b_E psi_E + c_E dH'
//   n'  = n + g + G n + mk sp,   sp = (E + E') . J' / 2
// Objective per step: phi = sum over the plane k = p (interior rectangle) of
// mx Hy'(k-1) - my Hx'(k-1), m = (E + E')/2: the +z Poynting flux (times
// dt dx^2 E0^2 / eta0 in joules).
//
// The reverse of step n maps the adjoints of x^{n+1} to those of x^n in the
// reverse order of the sub-steps.  Because the backward curl is the
// transpose of the forward curl, it has the structure of a Yee step run
// backwards, in three launches:
//   R1 (pointwise): objective and population terms, PEC mask, the eps
//      gradient, mu = ie lambda_E (the E update's coefficient field), the
//      Lorentz update's adjoint, the psi_E adjoint memories;
//   R2 (like the H pass, forward differences of mu): lambda_H, psi_H memories;
//   R3 (like the E pass, backward differences of lambda_H): lambda_E.
// The three use the forward states x^n and x^{n+1} kept by the segment store.
#include "mb_host.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <string>
#include <vector>

namespace mb {

namespace {

// Forward fields of one stored step: E, J, n1..n3 of every cell and Hx, Hy
// of the objective's H layer (k = z_plane - 1, indexed i + n_x j); P and the
// rest of H enter the reverse sweep only linearly.
struct FwdFields {
    const float *ex, *ey, *ez, *jx, *jy, *jz, *n1, *n2, *n3, *hpx, *hpy;
};

struct AdjArgs {
    DevGrid g;
    int L;
    const uint8_t* mat;
    const float* inv_eps;
    const float* lut_inv_eps;
    int n_lut;                  // at most two eps_r values: 1/eps_r of ids 0, 1 below
    float ie0, ie1;
    DevCpml pml;                // forward tables (psi pointers unused)
    float *lpsx, *lpsy, *lpsz;  // adjoint CPML memories, forward layout
    FwdFields x0, x1;           // states at n and n+1
    float *le, *lh, *lj, *lp, *ln, *mu;   // 3 arrays of ncell each
    double* geps;               // d phi / d eps per cell (device units)
    double* acc;                // [0, 64): objective slots, [64, 128): pump slots
    DevGain gain;
    float dg[3], dG[3][3], dmk[3];
    int zp, rx0, rx1, ry0, ry1;
    float S;
    const long long* n_ptr;     // index of the forward step being reversed (device)
};

constexpr int kAccSlots = 64;

__device__ __forceinline__ float ie_of(const AdjArgs& a, uint32_t c) {
    if (a.inv_eps) return __ldg(a.inv_eps + c);
    const int id = __ldg(a.mat + c) & 0x7f;
    return a.n_lut <= 2 ? (id ? a.ie1 : a.ie0) : __ldg(a.lut_inv_eps + id);
}

__device__ __forceinline__ bool in_slab(int i, int n, int L) { return L > 0 && (i < L || i >= n - L); }

// FP32 warp sum, one FP64 atomic per warp into a slot.
__device__ __forceinline__ void warp_acc(double* acc, float v, unsigned slot) {
    const unsigned full = 0xffffffffu;
    if (!__any_sync(full, v != 0.0f)) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc + (slot % kAccSlots), (double)v);
}

__device__ __forceinline__ unsigned block_slot() {
    return blockIdx.x + 7u * blockIdx.y + 13u * blockIdx.z + 3u * ((threadIdx.y * blockDim.x + threadIdx.x) >> 5);
}

// ------------------------------------------------------------------- R1
// Pointwise part of the reverse of the step (x0 -> x1) at cell (i, j, k),
// given lambda_E of x1 in l1x..l1z; returns the cell's objective and pump
// terms in obj, gw (zero for lanes outside the grid: valid false).
__device__ __forceinline__ void adj_point_cell(const AdjArgs& a, int i, int j, int k, bool valid,
                                               float l1x, float l1y, float l1z, float& obj, float& gw) {
    obj = 0.0f;
    gw = 0.0f;
    if (valid) {
        const uint32_t N = a.g.ncell;
        const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
        const float e0x = __ldcs(a.x0.ex + c), e0y = __ldcs(a.x0.ey + c), e0z = __ldcs(a.x0.ez + c);
        const float e1x = __ldcs(a.x1.ex + c), e1y = __ldcs(a.x1.ey + c), e1z = __ldcs(a.x1.ez + c);
        float l0x = 0.0f, l0y = 0.0f, l0z = 0.0f;
        // objective: mx Hy(k-1) - my Hx(k-1) on the plane k = zp
        if (k == a.zp && i >= a.rx0 && i < a.rx1 && j >= a.ry0 && j < a.ry1) {
            const uint32_t cp = (uint32_t)i + (uint32_t)a.g.nx * j;
            const float hxk = __ldcs(a.x1.hpx + cp), hyk = __ldcs(a.x1.hpy + cp);
            l1x += 0.5f * hyk;
            l1y -= 0.5f * hxk;
            l0x += 0.5f * hyk;
            l0y -= 0.5f * hxk;
            obj = 0.5f * (e0x + e1x) * hyk - 0.5f * (e0y + e1y) * hxk;
        }
        const uint8_t m = __ldg(a.mat + c);
        const bool gain = a.gain.on && (m & 0x80);
        float ljx = 0.0f, ljy = 0.0f, ljz = 0.0f;
        float j1x = 0.0f, j1y = 0.0f, j1z = 0.0f;
        float n1 = 0.0f, n2 = 0.0f, n3 = 0.0f, ln1 = 0.0f, ln2 = 0.0f, ln3 = 0.0f;
        if (gain) {
            // populations: n' = n + g + G n + mk sp
            j1x = __ldcs(a.x1.jx + c);
            j1y = __ldcs(a.x1.jy + c);
            j1z = __ldcs(a.x1.jz + c);
            n1 = __ldcs(a.x0.n1 + c);
            n2 = __ldcs(a.x0.n2 + c);
            n3 = __ldcs(a.x0.n3 + c);
            const float lq[3] = {a.ln[c], a.ln[c + N], a.ln[c + 2 * N]};
            const float sp = 0.5f * ((e0x + e1x) * j1x + (e0y + e1y) * j1y + (e0z + e1z) * j1z);
            const float nq[3] = {n1, n2, n3};
            float lsp = 0.0f;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                lsp += a.gain.mk[r] * lq[r];
                gw += lq[r] * (a.dg[r] + a.dG[r][0] * nq[0] + a.dG[r][1] * nq[1] + a.dG[r][2] * nq[2] +
                               a.dmk[r] * sp);
            }
            ln1 = lq[0] + a.gain.G[0][0] * lq[0] + a.gain.G[1][0] * lq[1] + a.gain.G[2][0] * lq[2];
            ln2 = lq[1] + a.gain.G[0][1] * lq[0] + a.gain.G[1][1] * lq[1] + a.gain.G[2][1] * lq[2];
            ln3 = lq[2] + a.gain.G[0][2] * lq[0] + a.gain.G[1][2] * lq[1] + a.gain.G[2][2] * lq[2];
            const float h = 0.5f * lsp;
            l1x += h * j1x;
            l1y += h * j1y;
            l1z += h * j1z;
            l0x += h * j1x;
            l0y += h * j1y;
            l0z += h * j1z;
            ljx = a.lj[c] + h * (e0x + e1x);
            ljy = a.lj[c + N] + h * (e0y + e1y);
            ljz = a.lj[c + 2 * N] + h * (e0z + e1z);
        }
        // E update: PEC mask, eps gradient, mu = ie lambda
        const float ltx = (j == 0 || k == 0) ? 0.0f : l1x;
        const float lty = (i == 0 || k == 0) ? 0.0f : l1y;
        const float ltz = (i == 0 || j == 0) ? 0.0f : l1z;
        const float ie = ie_of(a, c);
        const float ge = -ie * (ltx * (e1x - e0x) + lty * (e1y - e0y) + ltz * (e1z - e0z));
        if (ge != 0.0f) a.geps[c] += (double)ge;
        l0x += ltx;
        l0y += lty;
        l0z += ltz;
        const float ux = ie * ltx, uy = ie * lty, uz = ie * ltz;
        a.mu[c] = ux;
        a.mu[c + N] = uy;
        a.mu[c + 2 * N] = uz;
        // psi_E adjoint memories: lambda_tot = b lambda_prev + sign S u
        const int L = a.L, L2 = 2 * L, nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
        const float S = a.S;
        if (in_slab(i, nx, L)) {
            const uint32_t plane = (uint32_t)nz * ny * L2;
            const uint32_t q = ((uint32_t)k * ny + j) * L2 + slab_index(i, nx, L);
            const float b = __ldg(a.pml.bex + i);
            a.lpsx[q] = b * a.lpsx[q] - S * uy;                  // psi_yx (Ey, -)
            a.lpsx[q + plane] = b * a.lpsx[q + plane] + S * uz;  // psi_zx (Ez, +)
        }
        if (in_slab(j, ny, L)) {
            const uint32_t plane = (uint32_t)nz * L2 * nx;
            const uint32_t q = ((uint32_t)k * L2 + slab_index(j, ny, L)) * nx + i;
            const float b = __ldg(a.pml.bey + j);
            a.lpsy[q] = b * a.lpsy[q] + S * ux;                  // psi_xy (Ex, +)
            a.lpsy[q + plane] = b * a.lpsy[q + plane] - S * uz;  // psi_zy (Ez, -)
        }
        if (in_slab(k, nz, L)) {
            const uint32_t plane = (uint32_t)L2 * ny * nx;
            const uint32_t q = ((uint32_t)slab_index(k, nz, L) * ny + j) * nx + i;
            const float b = __ldg(a.pml.bez + k);
            a.lpsz[q] = b * a.lpsz[q] - S * ux;                  // psi_xz (Ex, -)
            a.lpsz[q + plane] = b * a.lpsz[q + plane] + S * uy;  // psi_yz (Ey, +)
        }
        // Lorentz update: J' = cJ1 J + cJE dn E - cJP P + amp(n2) zeta, P' = P + J'
        if (gain) {
            const float tx = ljx - ux + a.lp[c];
            const float ty = ljy - uy + a.lp[c + N];
            const float tz = ljz - uz + a.lp[c + 2 * N];
            const DevGain& G = a.gain;
            a.lp[c] -= G.cJP * tx;
            a.lp[c + N] -= G.cJP * ty;
            a.lp[c + 2 * N] -= G.cJP * tz;
            a.lj[c] = G.cJ1 * tx;
            a.lj[c + N] = G.cJ1 * ty;
            a.lj[c + 2 * N] = G.cJ1 * tz;
            const float kE = G.cJE * (n1 - n2);
            l0x += kE * tx;
            l0y += kE * ty;
            l0z += kE * tz;
            const float ldn = G.cJE * (e0x * tx + e0y * ty + e0z * tz);
            float z0, z1, z2;
            langevin_normals(c, (uint32_t)*a.n_ptr, G.key0, G.key1, z0, z1, z2);
            const float damp = n2 > 0.0f ? 0.5f * G.cJN * rsqrtf(n2 + G.nfloor) : 0.0f;
            a.ln[c] = ln1 + ldn;
            a.ln[c + N] = ln2 - ldn + damp * (z0 * tx + z1 * ty + z2 * tz);
            a.ln[c + 2 * N] = ln3;
        }
        a.le[c] = l0x;
        a.le[c + N] = l0y;
        a.le[c + 2 * N] = l0z;
    }
}

__global__ void __launch_bounds__(256) k_adj_point(AdjArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const bool valid = i < a.g.nx && j < a.g.ny;
    float l1x = 0.0f, l1y = 0.0f, l1z = 0.0f;
    if (valid) {
        const uint32_t N = a.g.ncell;
        const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
        l1x = a.le[c];
        l1y = a.le[c + N];
        l1z = a.le[c + 2 * N];
    }
    float obj, gw;
    adj_point_cell(a, i, j, k, valid, l1x, l1y, l1z, obj, gw);
    const unsigned slot = block_slot();
    warp_acc(a.acc, obj, slot);
    warp_acc(a.acc + kAccSlots, gw, slot);
}

// ------------------------------------------------------------------- R2
// W_ab(c): coefficient of the backward difference along b in E_a's update
// (S mu_a with the curl's sign, plus c_E times the psi_E adjoint memory).
struct WCoef {
    float xy, xz, yz, yx, zx, zy;
};

__device__ __forceinline__ float lpsi_x(const AdjArgs& a, const float* p, int f, int i, int j, int k) {
    const int L2 = 2 * a.L;
    const uint32_t plane = (uint32_t)a.g.nz * a.g.ny * L2;
    return p[f * plane + ((uint32_t)k * a.g.ny + j) * L2 + slab_index(i, a.g.nx, a.L)];
}
__device__ __forceinline__ float lpsi_y(const AdjArgs& a, const float* p, int f, int i, int j, int k) {
    const int L2 = 2 * a.L;
    const uint32_t plane = (uint32_t)a.g.nz * L2 * a.g.nx;
    return p[f * plane + ((uint32_t)k * L2 + slab_index(j, a.g.ny, a.L)) * a.g.nx + i];
}
__device__ __forceinline__ float lpsi_z(const AdjArgs& a, const float* p, int f, int i, int j, int k) {
    const int L2 = 2 * a.L;
    const uint32_t plane = (uint32_t)L2 * a.g.ny * a.g.nx;
    return p[f * plane + ((uint32_t)slab_index(k, a.g.nz, a.L) * a.g.ny + j) * a.g.nx + i];
}

// Coefficients at cell (i, j, k) (zero outside the grid).
__device__ __forceinline__ WCoef w_coef(const AdjArgs& a, int i, int j, int k) {
    WCoef w{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i >= a.g.nx || j >= a.g.ny || k >= a.g.nz) return w;
    const uint32_t N = a.g.ncell;
    const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
    const float S = a.S;
    const float ux = a.mu[c], uy = a.mu[c + N], uz = a.mu[c + 2 * N];
    w.xy = S * ux;
    w.xz = -S * ux;
    w.yz = S * uy;
    w.yx = -S * uy;
    w.zx = S * uz;
    w.zy = -S * uz;
    const int L = a.L;
    if (in_slab(i, a.g.nx, L)) {
        const float cc = __ldg(a.pml.cex + i);
        w.yx += cc * lpsi_x(a, a.lpsx, 0, i, j, k);
        w.zx += cc * lpsi_x(a, a.lpsx, 1, i, j, k);
    }
    if (in_slab(j, a.g.ny, L)) {
        const float cc = __ldg(a.pml.cey + j);
        w.xy += cc * lpsi_y(a, a.lpsy, 0, i, j, k);
        w.zy += cc * lpsi_y(a, a.lpsy, 1, i, j, k);
    }
    if (in_slab(k, a.g.nz, L)) {
        const float cc = __ldg(a.pml.cez + k);
        w.xz += cc * lpsi_z(a, a.lpsz, 0, i, j, k);
        w.yz += cc * lpsi_z(a, a.lpsz, 1, i, j, k);
    }
    return w;
}

// The coefficients of an interior cell (no CPML memory): S mu with the curl's signs.
__device__ __forceinline__ WCoef w_plain(float S, float ux, float uy, float uz) {
    WCoef w;
    w.xy = S * ux;
    w.xz = -S * ux;
    w.yz = S * uy;
    w.yx = -S * uy;
    w.zx = S * uz;
    w.zy = -S * uz;
    return w;
}

__global__ void __launch_bounds__(256) k_adj_h(AdjArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const int nx = a.g.nx, ny = a.g.ny, nz = a.g.nz, L = a.L;
    const bool valid = i < nx && j < ny;
    // a warp none of whose cells or +1 neighbours lies in a CPML slab takes
    // the coefficients without the memories (the same values)
    const bool pml = __any_sync(0xffffffffu, valid && (in_slab(i, nx, L) || in_slab(i + 1, nx, L) ||
                                                       in_slab(j, ny, L) || in_slab(j + 1, ny, L) ||
                                                       in_slab(k, nz, L) || in_slab(k + 1, nz, L)));
    if (!valid) return;
    const uint32_t N = a.g.ncell;
    const uint32_t c = (uint32_t)i + (uint32_t)nx * j + a.g.nxy * k;
    float hx = a.lh[c], hy = a.lh[c + N], hz = a.lh[c + 2 * N];
    // objective: H sites of the layer k = zp - 1
    if (k + 1 == a.zp && i >= a.rx0 && i < a.rx1 && j >= a.ry0 && j < a.ry1) {
        const uint32_t cu = c + a.g.nxy;
        hy += 0.5f * (__ldcs(a.x0.ex + cu) + __ldcs(a.x1.ex + cu));
        hx -= 0.5f * (__ldcs(a.x0.ey + cu) + __ldcs(a.x1.ey + cu));
    }
    WCoef w0, wi, wj, wk;
    if (!pml) {
        const float S = a.S;
        w0 = w_plain(S, a.mu[c], a.mu[c + N], a.mu[c + 2 * N]);
        wi = wj = wk = WCoef{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (i + 1 < nx) {
            wi.yx = -S * a.mu[c + 1 + N];
            wi.zx = S * a.mu[c + 1 + 2 * N];
        }
        if (j + 1 < ny) {
            wj.xy = S * a.mu[c + nx];
            wj.zy = -S * a.mu[c + nx + 2 * N];
        }
        if (k + 1 < nz) {
            wk.xz = -S * a.mu[c + a.g.nxy];
            wk.yz = S * a.mu[c + a.g.nxy + N];
        }
    } else {
        w0 = w_coef(a, i, j, k);
        wi = w_coef(a, i + 1, j, k);
        wj = w_coef(a, i, j + 1, k);
        wk = w_coef(a, i, j, k + 1);
    }
    hz += (w0.xy - wj.xy) + (w0.yx - wi.yx);
    hy += (w0.xz - wk.xz) + (w0.zx - wi.zx);
    hx += (w0.yz - wk.yz) + (w0.zy - wj.zy);
    a.lh[c] = hx;
    a.lh[c + N] = hy;
    a.lh[c + 2 * N] = hz;
    if (!pml) return;
    // psi_H adjoint memories: lambda_tot = b lambda_prev - sign S lambda_H
    const int L2 = 2 * L;
    const float S = a.S;
    if (in_slab(i, nx, L)) {
        const uint32_t plane = (uint32_t)nz * ny * L2;
        const uint32_t q = ((uint32_t)k * ny + j) * L2 + slab_index(i, nx, L);
        const float b = __ldg(a.pml.bhx + i);
        a.lpsx[q + 2 * plane] = b * a.lpsx[q + 2 * plane] + S * hy;   // psi_yx (Hy, -)
        a.lpsx[q + 3 * plane] = b * a.lpsx[q + 3 * plane] - S * hz;   // psi_zx (Hz, +)
    }
    if (in_slab(j, ny, L)) {
        const uint32_t plane = (uint32_t)nz * L2 * nx;
        const uint32_t q = ((uint32_t)k * L2 + slab_index(j, ny, L)) * nx + i;
        const float b = __ldg(a.pml.bhy + j);
        a.lpsy[q + 2 * plane] = b * a.lpsy[q + 2 * plane] - S * hx;   // psi_xy (Hx, +)
        a.lpsy[q + 3 * plane] = b * a.lpsy[q + 3 * plane] + S * hz;   // psi_zy (Hz, -)
    }
    if (in_slab(k, nz, L)) {
        const uint32_t plane = (uint32_t)L2 * ny * nx;
        const uint32_t q = ((uint32_t)slab_index(k, nz, L) * ny + j) * nx + i;
        const float b = __ldg(a.pml.bhz + k);
        a.lpsz[q + 2 * plane] = b * a.lpsz[q + 2 * plane] + S * hx;   // psi_xz (Hx, -)
        a.lpsz[q + 3 * plane] = b * a.lpsz[q + 3 * plane] - S * hy;   // psi_yz (Hy, +)
    }
}

// ------------------------------------------------------------------- R3
// V_ab(c): coefficient of the forward difference along b in H_a's update
// (-S lambda_Ha with the curl's sign, plus c_H times the psi_H memory).
__device__ __forceinline__ WCoef v_coef(const AdjArgs& a, int i, int j, int k) {
    WCoef v{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < 0 || j < 0 || k < 0) return v;
    const uint32_t N = a.g.ncell;
    const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
    const float S = a.S;
    const float hx = a.lh[c], hy = a.lh[c + N], hz = a.lh[c + 2 * N];
    v.xy = -S * hx;
    v.xz = S * hx;
    v.yz = -S * hy;
    v.yx = S * hy;
    v.zx = -S * hz;
    v.zy = S * hz;
    const int L = a.L;
    if (in_slab(i, a.g.nx, L)) {
        const float cc = __ldg(a.pml.chx + i);
        v.yx += cc * lpsi_x(a, a.lpsx, 2, i, j, k);
        v.zx += cc * lpsi_x(a, a.lpsx, 3, i, j, k);
    }
    if (in_slab(j, a.g.ny, L)) {
        const float cc = __ldg(a.pml.chy + j);
        v.xy += cc * lpsi_y(a, a.lpsy, 2, i, j, k);
        v.zy += cc * lpsi_y(a, a.lpsy, 3, i, j, k);
    }
    if (in_slab(k, a.g.nz, L)) {
        const float cc = __ldg(a.pml.chz + k);
        v.xz += cc * lpsi_z(a, a.lpsz, 2, i, j, k);
        v.yz += cc * lpsi_z(a, a.lpsz, 3, i, j, k);
    }
    return v;
}

// The coefficients of an interior cell (no CPML memory): -S lambda_H with the curl's signs.
__device__ __forceinline__ WCoef v_plain(float S, float hx, float hy, float hz) {
    WCoef v;
    v.xy = -S * hx;
    v.xz = S * hx;
    v.yz = -S * hy;
    v.yx = S * hy;
    v.zx = -S * hz;
    v.zy = S * hz;
    return v;
}

// The lane's cell or one of its -1 neighbours lies in a CPML slab.
__device__ __forceinline__ bool near_slab_lo(const AdjArgs& a, int i, int j, int k) {
    const int L = a.L;
    return in_slab(i, a.g.nx, L) || in_slab(i - 1, a.g.nx, L) || in_slab(j, a.g.ny, L) ||
           in_slab(j - 1, a.g.ny, L) || in_slab(k, a.g.nz, L) || in_slab(k - 1, a.g.nz, L);
}

// lambda_E of x^n at cell (i, j, k): the partial value left in le by R1 plus
// the transposed H update (backward differences of the V coefficients).
// pml false (the whole warp away from the CPML slabs): the coefficients
// without the memories, the same values.
__device__ __forceinline__ void adj_e_gather(const AdjArgs& a, int i, int j, int k, uint32_t c, bool pml,
                                             float& lx, float& ly, float& lz) {
    const uint32_t N = a.g.ncell;
    WCoef v0, vi, vj, vk;
    if (!pml) {
        const float S = a.S;
        const uint32_t nx = a.g.nx, nxy = a.g.nxy;
        v0 = v_plain(S, a.lh[c], a.lh[c + N], a.lh[c + 2 * N]);
        vi = vj = vk = WCoef{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (i >= 1) {
            vi.zx = -S * a.lh[c - 1 + 2 * N];
            vi.yx = S * a.lh[c - 1 + N];
        }
        if (j >= 1) {
            vj.zy = S * a.lh[c - nx + 2 * N];
            vj.xy = -S * a.lh[c - nx];
        }
        if (k >= 1) {
            vk.yz = -S * a.lh[c - nxy + N];
            vk.xz = S * a.lh[c - nxy];
        }
    } else {
        v0 = v_coef(a, i, j, k);
        vi = v_coef(a, i - 1, j, k);
        vj = v_coef(a, i, j - 1, k);
        vk = v_coef(a, i, j, k - 1);
    }
    lx = a.le[c] + ((vk.yz - v0.yz) + (vj.zy - v0.zy));
    ly = a.le[c + N] + ((vk.xz - v0.xz) + (vi.zx - v0.zx));
    lz = a.le[c + 2 * N] + ((vj.xy - v0.xy) + (vi.yx - v0.yx));
}

__global__ void __launch_bounds__(256) k_adj_e(AdjArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= a.g.nx || j >= a.g.ny) return;
    const uint32_t N = a.g.ncell;
    const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
    float lx, ly, lz;
    adj_e_gather(a, i, j, k, c, true, lx, ly, lz);
    a.le[c] = lx;
    a.le[c + N] = ly;
    a.le[c + 2 * N] = lz;
}

// R3 of step n fused with R1 of step n - 1 (a's x0, x1, n_ptr describe
// step n - 1): lambda_E of x^n stays in registers.  R3 reads lambda_H and the
// psi_H memories of neighbours, which R1 does not write.  Bounded to 40
// registers (6 blocks per SM, a few spilled bytes): the launch is latency
// bound, and the added warps gain more than the spills cost.
__global__ void __launch_bounds__(256, 6) k_adj_e_point(AdjArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const bool valid = i < a.g.nx && j < a.g.ny;
    const bool pml = __any_sync(0xffffffffu, valid && near_slab_lo(a, i, j, k));
    float lx = 0.0f, ly = 0.0f, lz = 0.0f;
    if (valid) adj_e_gather(a, i, j, k, (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k, pml, lx, ly, lz);
    float obj, gw;
    adj_point_cell(a, i, j, k, valid, lx, ly, lz, obj, gw);
    const unsigned slot = block_slot();
    warp_acc(a.acc, obj, slot);
    warp_acc(a.acc + kAccSlots, gw, slot);
}

// Store slot of one step: E (arrays 0..2) and J, n1..n3 (arrays 9..14) of
// the field block, Hx and Hy of plane kp, and the step counter.  16-byte
// moves when n_cells and the plane size are multiples of 4 (every array then
// starts 16-byte aligned).  The stores are marked streaming (evict first), so
// the segment store (gigabytes) does not push the recomputed state out of
// L2; the reverse kernels read the stored states the same way.
__global__ void k_keep(const float* __restrict__ F, float* __restrict__ dst, uint32_t n,
                       uint32_t nxy, int kp, const long long* __restrict__ ctr,
                       long long* __restrict__ slot_n) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *slot_n = *ctr;
    const size_t n3 = 3 * (size_t)n, n6 = 6 * (size_t)n;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const float* hpx = F + 3 * (size_t)n + (size_t)nxy * kp;
    const float* hpy = F + 4 * (size_t)n + (size_t)nxy * kp;
    float* dp = dst + 9 * (size_t)n;
    if ((n & 3u) == 0 && (nxy & 3u) == 0) {
        const float4* a = reinterpret_cast<const float4*>(F);
        const float4* b = reinterpret_cast<const float4*>(F + 9 * (size_t)n);
        float4* d = reinterpret_cast<float4*>(dst);
        for (size_t t = t0; t < n3 / 4; t += stride) __stcs(d + t, a[t]);
        for (size_t t = t0; t < n6 / 4; t += stride) __stcs(d + n3 / 4 + t, b[t]);
        for (size_t t = t0; t < nxy / 4; t += stride) {
            __stcs(reinterpret_cast<float4*>(dp) + t, reinterpret_cast<const float4*>(hpx)[t]);
            __stcs(reinterpret_cast<float4*>(dp + nxy) + t, reinterpret_cast<const float4*>(hpy)[t]);
        }
    } else {
        const float* b = F + 9 * (size_t)n;
        for (size_t t = t0; t < n3; t += stride) __stcs(dst + t, F[t]);
        for (size_t t = t0; t < n6; t += stride) __stcs(dst + n3 + t, b[t]);
        for (size_t t = t0; t < nxy; t += stride) {
            __stcs(dp + t, hpx[t]);
            __stcs(dp + nxy + t, hpy[t]);
        }
    }
}

// Output: grad[c] = scale * geps[c].
__global__ void k_adj_out(const double* geps, float* out, uint32_t n, double scale) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        out[c] = (float)(scale * geps[c]);
}

}  // namespace

}  // namespace mb

namespace {

struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
};

int afail(mb_ctx* c, int code, const std::string& msg) {
    c->err = msg;
    mb::set_thread_error(msg);
    return code;
}

#define MB_ACUDA(c, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            rc = afail((c), e_ == cudaErrorMemoryAllocation ? MB_ERR_OOM : MB_ERR_CUDA,    \
                       std::string(#call) + ": " + cudaGetErrorString(e_));                \
            goto done;                                                                     \
        }                                                                                  \
    } while (0)

}  // namespace

extern "C" int mb_adjoint_energy_zface(mb_ctx* c, int n_steps, int ckpt_every, int z_plane,
                                       float* d_grad_eps, double* grad_pump, double* J_out) {
    if (!c) {
        mb::set_thread_error("null context");
        return MB_ERR_ARG;
    }
    mb::join_probes(c);
    if (n_steps < 1) return afail(c, MB_ERR_ARG, "n_steps must be >= 1");
    if (!c->have_material) return afail(c, MB_ERR_STATE, "no material set");
    if (c->slab) return afail(c, MB_ERR_STATE, "the adjoint runs on a whole grid, not on a z-slab");
    const int zp = z_plane < 0 ? c->args.flux.phi[2] : z_plane;
    if (zp < 1 || zp >= c->nz) return afail(c, MB_ERR_ARG, "z plane must satisfy 1 <= p < n_z");
    const int K = std::min(ckpt_every > 0 ? ckpt_every : 200, n_steps);
    const int nseg = (n_steps + K - 1) / K;
    const size_t N = (size_t)c->ncell;
    const size_t sb = mb::state_device_bytes(c);
    const size_t nxy = (size_t)c->nx * c->ny;
    const size_t slot = 9 * N + 2 * nxy;   // floats per stored step: E, J, n1..n3, Hx/Hy of one plane
    const size_t psi_total = c->psi_elems[0] + c->psi_elems[1] + c->psi_elems[2];
    NvtxScope range("mb_adjoint_energy_zface");
    // the sweeps below step the context in place (state in its own arrays)
    const bool was_single_pass = mb::hold_in_place(c);

    int rc = MB_OK;
    char* ckpt = nullptr;
    float* store = nullptr;
    float* adj = nullptr;
    double* geps = nullptr;
    double* acc = nullptr;
    long long* slot_n = nullptr;
    cudaGraphExec_t seg_graph = nullptr;
    bool graph_ok = true;
    mb::AdjArgs a{};
    mb::StepArgs fa = c->args;
    // launch shapes of the recomputation (tuned below for its own regime)
    mb::PassTune th = c->tune_h, te_r = c->tune_e;
    auto maps_for = [&](const mb::PassTune& t) -> const mb::TmaMaps* {
        return t.variant == mb::kVariantTma ? mb::tma_maps(c, t) : nullptr;
    };
    double acc_h[2 * mb::kAccSlots];
    const dim3 blk(32, 8, 1);
    const dim3 grd((c->nx + 31) / 32, (c->ny + 7) / 8, c->nz);
    const float* F = c->d_fields;

    // keep(t): the context's E, J, n1..n3, the objective's H layer and the
    // step counter into store slot t
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int keep_blocks = (int)std::max<size_t>(1, std::min<size_t>((6 * N / 4 + 255) / 256, (size_t)sms * 8));
    auto keep = [&](int t) -> cudaError_t {
        mb::k_keep<<<keep_blocks, 256, 0, c->stream>>>(F, store + slot * t, (uint32_t)N, (uint32_t)nxy,
                                                       zp - 1, c->d_ctr, slot_n + t);
        return cudaGetLastError();
    };
    auto step_args = [&](int t) {
        auto fields = [&](int q) {
            const float* b = store + slot * q;
            return mb::FwdFields{b, b + N, b + 2 * N, b + 3 * N, b + 4 * N, b + 5 * N,
                                 b + 6 * N, b + 7 * N, b + 8 * N, b + 9 * N, b + 9 * N + nxy};
        };
        a.x0 = fields(t);
        a.x1 = fields(t + 1);
        a.n_ptr = slot_n + t;
    };
    // the reverse of stored steps len-1 .. 0: R1, then per step R2 and R3
    // fused with the next step's R1
    auto reverse = [&](int len) -> cudaError_t {
        step_args(len - 1);
        mb::k_adj_point<<<grd, blk, 0, c->stream>>>(a);
        for (int t = len - 1; t >= 0; --t) {
            mb::k_adj_h<<<grd, blk, 0, c->stream>>>(a);
            if (t > 0) {
                step_args(t - 1);
                mb::k_adj_e_point<<<grd, blk, 0, c->stream>>>(a);
            } else {
                mb::k_adj_e<<<grd, blk, 0, c->stream>>>(a);
            }
        }
        return cudaGetLastError();
    };
    // recompute a segment from the checkpoint restored into the context
    // (same pass kernels, probes and flux off), keeping every state
    auto recompute = [&](int len) -> cudaError_t {
        cudaError_t e = keep(0);
        for (int t = 0; t < len && e == cudaSuccess; ++t) {
            mb::launch_h_pass(fa, th, maps_for(th), c->stream);
            mb::launch_e_pass(fa, te_r, maps_for(te_r), c->stream);
            e = keep(t + 1);
        }
        return e;
    };

    MB_ACUDA(c, cudaMalloc((void**)&ckpt, sb * (nseg + 1)));
    MB_ACUDA(c, cudaMalloc((void**)&store, sizeof(float) * slot * (K + 1)));
    MB_ACUDA(c, cudaMalloc((void**)&adj, sizeof(float) * (18 * N + psi_total)));
    MB_ACUDA(c, cudaMalloc((void**)&geps, sizeof(double) * N));
    MB_ACUDA(c, cudaMalloc((void**)&acc, sizeof(double) * 2 * mb::kAccSlots));
    MB_ACUDA(c, cudaMalloc((void**)&slot_n, sizeof(long long) * (K + 1)));

    // forward sweep: a checkpoint at the start of every segment but the last,
    // whose states are kept as it runs (it is reversed first)
    for (int m = 0; m + 1 < nseg; ++m) {
        if ((rc = mb::state_snapshot(c, ckpt + sb * m))) goto done;
        if ((rc = mb_step(c, K))) goto done;
    }
    fa.flux.on = 0;
    if (nseg > 1) {
        // The recomputation streams from HBM (the segment store evicts the
        // state from L2), unlike the plain step the context was tuned for:
        // time candidate shapes in its own sequence (store, H, E) from the
        // start of the last segment, then put the state back (the store is
        // still empty).
        if ((rc = mb::state_snapshot(c, ckpt + sb * (nseg - 1)))) goto done;
        std::vector<mb::PassTune> cand = {c->tune_h, c->tune_e};
        for (int kz : {4, 8, 16}) cand.push_back({mb::kVariantZmarch, dim3(32, 4, 1), kz});
        cand.push_back({mb::kVariantZmarch, dim3(32, 8, 1), 8});
        cand.push_back({mb::kVariantZmarch, dim3(64, 4, 1), 8});
        if (mb::tma_e_supported(fa))
            for (dim3 b : {dim3(32, 4, 1), dim3(64, 4, 1), dim3(32, 8, 1)})
                for (int kz : {4, 8, 16}) cand.push_back({mb::kVariantTma, b, kz});
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int pass = 0; pass < 2; ++pass) {
            float best = 1e30f;
            mb::PassTune pick = pass == 0 ? th : te_r;
            for (const mb::PassTune& t : cand) {
                if (t.kz > 2 * c->nz || (t.variant == mb::kVariantTma && !maps_for(t))) continue;
                float tot = 0.0f;
                for (int r = 0; r < 3; ++r) {
                    MB_ACUDA(c, keep(0));
                    if (pass == 1) mb::launch_h_pass(fa, th, maps_for(th), c->stream);
                    cudaEventRecord(e0, c->stream);
                    if (pass == 0) mb::launch_h_pass(fa, t, maps_for(t), c->stream);
                    else mb::launch_e_pass(fa, t, maps_for(t), c->stream);
                    cudaEventRecord(e1, c->stream);
                    if (pass == 0) mb::launch_e_pass(fa, te_r, maps_for(te_r), c->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (r > 0) tot += ms;
                }
                if (tot < best) {
                    best = tot;
                    pick = t;
                }
            }
            if (pass == 0) th = pick;
            else te_r = pick;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        MB_ACUDA(c, cudaGetLastError());
        if ((rc = mb::state_restore(c, ckpt + sb * (nseg - 1)))) goto done;
    }

    {
        const int len = n_steps - (nseg - 1) * K;
        MB_ACUDA(c, keep(0));
        for (int t = 0; t < len; ++t) {
            MB_ACUDA(c, mb::enqueue_step(c));
            MB_ACUDA(c, keep(t + 1));
        }
    }
    if ((rc = mb::state_snapshot(c, ckpt + sb * nseg))) goto done;

    MB_ACUDA(c, cudaMemsetAsync(adj, 0, sizeof(float) * (18 * N + psi_total), c->stream));
    MB_ACUDA(c, cudaMemsetAsync(geps, 0, sizeof(double) * N, c->stream));
    MB_ACUDA(c, cudaMemsetAsync(acc, 0, sizeof(double) * 2 * mb::kAccSlots, c->stream));

    a.g = c->args.g;
    a.L = c->p.npml;
    a.mat = c->d_mat;
    a.inv_eps = c->args.f.inv_eps;
    a.lut_inv_eps = c->args.f.lut_inv_eps;
    a.n_lut = c->args.f.n_lut;
    a.ie0 = c->args.f.ie0;
    a.ie1 = c->args.f.ie1;
    a.pml = c->args.pml;
    a.lpsx = adj + 18 * N;
    a.lpsy = a.lpsx + c->psi_elems[0];
    a.lpsz = a.lpsy + c->psi_elems[1];
    a.le = adj;
    a.lh = adj + 3 * N;
    a.lj = adj + 6 * N;
    a.lp = adj + 9 * N;
    a.ln = adj + 12 * N;
    a.mu = adj + 15 * N;
    a.geps = geps;
    a.acc = acc;
    a.gain = c->args.gain;
    mb::gain_pump_derivative(c, a.dg, a.dG, a.dmk);
    a.zp = zp;
    a.rx0 = c->args.flux.r0[0];
    a.rx1 = c->args.flux.r1[0];
    a.ry0 = c->args.flux.r0[1];
    a.ry1 = c->args.flux.r1[1];
    a.S = c->args.S;

    // the last segment is in the store already
    MB_ACUDA(c, reverse(n_steps - (nseg - 1) * K));
    for (int m = nseg - 2; m >= 0; --m) {
        if ((rc = mb::state_restore(c, ckpt + sb * m))) goto done;
        if (graph_ok && !seg_graph) {
            // every earlier segment is full and repeats the same launches:
            // capture recomputation + reverse once
            cudaGraph_t g = nullptr;
            graph_ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (graph_ok) {
                cudaError_t le = recompute(K);
                if (le == cudaSuccess) le = reverse(K);
                const cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
                graph_ok = le == cudaSuccess && ce == cudaSuccess &&
                           cudaGraphInstantiate(&seg_graph, g, 0) == cudaSuccess;
                if (g) cudaGraphDestroy(g);
            }
            if (!graph_ok) {
                cudaGetLastError();
                if (seg_graph) cudaGraphExecDestroy(seg_graph);
                seg_graph = nullptr;
            }
        }
        if (seg_graph) {
            MB_ACUDA(c, cudaGraphLaunch(seg_graph, c->stream));
        } else {
            MB_ACUDA(c, recompute(K));
            MB_ACUDA(c, reverse(K));
        }
    }
    // back to the state after the forward sweep
    if ((rc = mb::state_restore(c, ckpt + sb * nseg))) goto done;
    {
        const double KJ = c->dt * c->E0 * (c->E0 / c->eta0) * c->dx * c->dx;
        if (d_grad_eps) {
            const int blocks = (int)std::min<size_t>((N + 255) / 256, 4096);
            mb::k_adj_out<<<blocks, 256, 0, c->stream>>>(geps, d_grad_eps, (uint32_t)N, KJ);
            MB_ACUDA(c, cudaGetLastError());
        }
        MB_ACUDA(c, cudaMemcpyAsync(acc_h, acc, sizeof(acc_h), cudaMemcpyDeviceToHost, c->stream));
        MB_ACUDA(c, cudaStreamSynchronize(c->stream));
        double sJ = 0.0, sW = 0.0;
        for (int q = 0; q < mb::kAccSlots; ++q) {
            sJ += acc_h[q];
            sW += acc_h[mb::kAccSlots + q];
        }
        if (J_out) *J_out = KJ * sJ;
        if (grad_pump) *grad_pump = KJ * sW;
    }
done:
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (seg_graph) cudaGraphExecDestroy(seg_graph);
    void* bufs[] = {ckpt, store, adj, geps, acc, slot_n};
    for (void* p : bufs)
        if (p) cudaFree(p);
    mb::restore_single_pass(c, was_single_pass);
    return rc;
}
