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

#include <algorithm>
#include <string>
#include <vector>

namespace mb {

namespace {

// Forward fields of one stored step (P is not needed by the reverse sweep).
struct FwdFields {
    const float *ex, *ey, *ez, *hx, *hy, *hz, *jx, *jy, *jz, *n1, *n2, *n3;
};

struct AdjArgs {
    DevGrid g;
    int L;
    const uint8_t* mat;
    const float* inv_eps;
    const float* lut_inv_eps;
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
    return a.inv_eps ? __ldg(a.inv_eps + c) : __ldg(a.lut_inv_eps + (__ldg(a.mat + c) & 0x7f));
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
__global__ void __launch_bounds__(256) k_adj_point(AdjArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    const bool valid = i < a.g.nx && j < a.g.ny;
    float obj = 0.0f, gw = 0.0f;
    if (valid) {
        const uint32_t N = a.g.ncell;
        const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
        const float e0x = __ldg(a.x0.ex + c), e0y = __ldg(a.x0.ey + c), e0z = __ldg(a.x0.ez + c);
        const float e1x = __ldg(a.x1.ex + c), e1y = __ldg(a.x1.ey + c), e1z = __ldg(a.x1.ez + c);
        float l1x = a.le[c], l1y = a.le[c + N], l1z = a.le[c + 2 * N];
        float l0x = 0.0f, l0y = 0.0f, l0z = 0.0f;
        // objective: mx Hy(k-1) - my Hx(k-1) on the plane k = zp
        if (k == a.zp && i >= a.rx0 && i < a.rx1 && j >= a.ry0 && j < a.ry1) {
            const float hxk = __ldg(a.x1.hx + c - a.g.nxy), hyk = __ldg(a.x1.hy + c - a.g.nxy);
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
            j1x = __ldg(a.x1.jx + c);
            j1y = __ldg(a.x1.jy + c);
            j1z = __ldg(a.x1.jz + c);
            n1 = __ldg(a.x0.n1 + c);
            n2 = __ldg(a.x0.n2 + c);
            n3 = __ldg(a.x0.n3 + c);
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

__global__ void __launch_bounds__(256) k_adj_h(AdjArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= a.g.nx || j >= a.g.ny) return;
    const uint32_t N = a.g.ncell;
    const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
    float hx = a.lh[c], hy = a.lh[c + N], hz = a.lh[c + 2 * N];
    // objective: H sites of the layer k = zp - 1
    if (k + 1 == a.zp && i >= a.rx0 && i < a.rx1 && j >= a.ry0 && j < a.ry1) {
        const uint32_t cu = c + a.g.nxy;
        hy += 0.5f * (__ldg(a.x0.ex + cu) + __ldg(a.x1.ex + cu));
        hx -= 0.5f * (__ldg(a.x0.ey + cu) + __ldg(a.x1.ey + cu));
    }
    const WCoef w0 = w_coef(a, i, j, k);
    const WCoef wi = w_coef(a, i + 1, j, k);
    const WCoef wj = w_coef(a, i, j + 1, k);
    const WCoef wk = w_coef(a, i, j, k + 1);
    hz += (w0.xy - wj.xy) + (w0.yx - wi.yx);
    hy += (w0.xz - wk.xz) + (w0.zx - wi.zx);
    hx += (w0.yz - wk.yz) + (w0.zy - wj.zy);
    a.lh[c] = hx;
    a.lh[c + N] = hy;
    a.lh[c + 2 * N] = hz;
    // psi_H adjoint memories: lambda_tot = b lambda_prev - sign S lambda_H
    const int L = a.L, L2 = 2 * L, nx = a.g.nx, ny = a.g.ny, nz = a.g.nz;
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

__global__ void __launch_bounds__(256) k_adj_e(AdjArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= a.g.nx || j >= a.g.ny) return;
    const uint32_t N = a.g.ncell;
    const uint32_t c = (uint32_t)i + (uint32_t)a.g.nx * j + a.g.nxy * k;
    const WCoef v0 = v_coef(a, i, j, k);
    const WCoef vi = v_coef(a, i - 1, j, k);
    const WCoef vj = v_coef(a, i, j - 1, k);
    const WCoef vk = v_coef(a, i, j, k - 1);
    a.le[c] += (vk.yz - v0.yz) + (vj.zy - v0.zy);
    a.le[c + N] += (vk.xz - v0.xz) + (vi.zx - v0.zx);
    a.le[c + 2 * N] += (vj.xy - v0.xy) + (vi.yx - v0.yx);
}

// Output: grad[c] = scale * geps[c].
__global__ void k_adj_out(const double* geps, float* out, uint32_t n, double scale) {
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        out[c] = (float)(scale * geps[c]);
}

}  // namespace

}  // namespace mb

namespace {

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
    if (n_steps < 1) return afail(c, MB_ERR_ARG, "n_steps must be >= 1");
    if (!c->have_material) return afail(c, MB_ERR_STATE, "no material set");
    const int zp = z_plane < 0 ? c->args.flux.phi[2] : z_plane;
    if (zp < 1 || zp >= c->nz) return afail(c, MB_ERR_ARG, "z plane must satisfy 1 <= p < n_z");
    const int K = std::min(ckpt_every > 0 ? ckpt_every : 200, n_steps);
    const int nseg = (n_steps + K - 1) / K;
    const size_t N = (size_t)c->ncell;
    const size_t sb = mb::state_device_bytes(c);
    const size_t slot = 12 * N;   // floats per stored step: E, H, J, n1..n3
    size_t psi_total = c->psi_elems[0] + c->psi_elems[1] + c->psi_elems[2];

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
    mb::PassTune th = c->tune_h, te = c->tune_e;
    double acc_h[2 * mb::kAccSlots];
    const dim3 blk(32, 8, 1);
    const dim3 grd((c->nx + 31) / 32, (c->ny + 7) / 8, c->nz);

    MB_ACUDA(c, cudaMalloc((void**)&ckpt, sb * (nseg + 1)));
    MB_ACUDA(c, cudaMalloc((void**)&store, sizeof(float) * slot * (K + 1)));
    MB_ACUDA(c, cudaMalloc((void**)&adj, sizeof(float) * (18 * N + psi_total)));
    MB_ACUDA(c, cudaMalloc((void**)&geps, sizeof(double) * N));
    MB_ACUDA(c, cudaMalloc((void**)&acc, sizeof(double) * 2 * mb::kAccSlots));
    MB_ACUDA(c, cudaMalloc((void**)&slot_n, sizeof(long long) * (K + 1)));

    // forward sweep with a checkpoint at the start of every segment
    for (int m = 0; m < nseg; ++m) {
        if ((rc = mb::state_snapshot(c, ckpt + sb * m))) goto done;
        if ((rc = mb_step(c, std::min(K, n_steps - m * K)))) goto done;
    }
    if ((rc = mb::state_snapshot(c, ckpt + sb * nseg))) goto done;

    MB_ACUDA(c, cudaMemsetAsync(adj, 0, sizeof(float) * (18 * N + psi_total), c->stream));
    MB_ACUDA(c, cudaMemsetAsync(geps, 0, sizeof(double) * N, c->stream));
    MB_ACUDA(c, cudaMemsetAsync(acc, 0, sizeof(double) * 2 * mb::kAccSlots, c->stream));

    // recomputation: same per-cell arithmetic, no probes or flux
    fa.flux.on = 0;
    if (te.variant == mb::kVariantTma) te = mb::PassTune{mb::kVariantZmarch, dim3(32, 4, 1), 16};

    a.g = c->args.g;
    a.L = c->p.npml;
    a.mat = c->d_mat;
    a.inv_eps = c->args.f.inv_eps;
    a.lut_inv_eps = c->args.f.lut_inv_eps;
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

    {
        // One segment: recompute from its checkpoint (already restored into the
        // context), keeping every state and the step counter, then reverse it.
        const float* F = c->d_fields;
        auto enqueue_segment = [&](int len) -> cudaError_t {
            auto keep = [&](int t) -> cudaError_t {
                float* dst = store + slot * t;
                cudaError_t e = cudaMemcpyAsync(dst, F, sizeof(float) * 6 * N, cudaMemcpyDeviceToDevice,
                                                c->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(dst + 6 * N, F + 9 * N, sizeof(float) * 6 * N,
                                        cudaMemcpyDeviceToDevice, c->stream);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(slot_n + t, c->d_ctr, sizeof(long long), cudaMemcpyDeviceToDevice,
                                        c->stream);
                return e;
            };
            cudaError_t e = keep(0);
            for (int t = 0; t < len && e == cudaSuccess; ++t) {
                mb::launch_h_pass(fa, th, c->stream);
                mb::launch_e_pass(fa, te, nullptr, c->stream);
                e = keep(t + 1);
            }
            for (int t = len - 1; t >= 0 && e == cudaSuccess; --t) {
                auto fields = [&](int q) {
                    const float* b = store + slot * q;
                    return mb::FwdFields{b, b + N, b + 2 * N, b + 3 * N, b + 4 * N, b + 5 * N,
                                         b + 6 * N, b + 7 * N, b + 8 * N, b + 9 * N, b + 10 * N, b + 11 * N};
                };
                a.x0 = fields(t);
                a.x1 = fields(t + 1);
                a.n_ptr = slot_n + t;
                mb::k_adj_point<<<grd, blk, 0, c->stream>>>(a);
                mb::k_adj_h<<<grd, blk, 0, c->stream>>>(a);
                mb::k_adj_e<<<grd, blk, 0, c->stream>>>(a);
                e = cudaGetLastError();
            }
            return e;
        };
        for (int m = nseg - 1; m >= 0; --m) {
            const int s0 = m * K, len = std::min(K, n_steps - s0);
            if ((rc = mb::state_restore(c, ckpt + sb * m))) goto done;
            if (len == K && graph_ok && !seg_graph) {
                // full segments repeat the same launches: capture them once
                cudaGraph_t g = nullptr;
                graph_ok = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                if (graph_ok) {
                    const cudaError_t le = enqueue_segment(K);
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
            if (len == K && seg_graph) {
                MB_ACUDA(c, cudaGraphLaunch(seg_graph, c->stream));
            } else {
                MB_ACUDA(c, enqueue_segment(len));
            }
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
    return rc;
}
