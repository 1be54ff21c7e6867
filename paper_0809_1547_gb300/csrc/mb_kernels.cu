// Probe, read-out and diagnostic kernels of the Maxwell–Bloch FDTD step
// (the two field passes live in mb_passes.cu):
//
//   k_point_dft   running DFT of E at the point probes (FP64 accumulators)
//   k_face_dft    running DFT of tangential E and H on the face sub-grids
//   k_plane_dft   running DFT of E on a whole z-plane (mode maps)
//   k_plane_energy  energy density of the cells of a z-plane (snapshots)
//   k_energy_*    two-pass deterministic reduction of the field energy
//   k_philox      the noise generator on given counters
//
// The probes run after the E pass of step n, whose last block has already
// advanced the step counter to n + 1: E^{n+1} is sampled at t_{n+1}.
#include "mb_host.h"

#include <cstdio>

namespace mb {

// Blocks (probe, group of 32 bins), a thread per bin (the phase factors of
// the bins spread over several SMs):
// acc[p][c][k] += E_c(t_{n+1}) exp(i w_k t_{n+1})   (scaled; times dt E0 on read-out)
__global__ void __launch_bounds__(32) k_point_dft(DevPointProbes pp, const float* ex, const float* ey,
                                                  const float* ez, const long long* step_ctr, double dt) {
    point_dft_block(pp, blockIdx.x, ex, ey, ez, step_ctr[0], dt,   // counter = n + 1
                    blockIdx.y * 32, gridDim.y * 32);
}

// Face DFT: block (chunk of points, face).  The block first forms the
// phase factors exp(i w_k t) of every bin at the E and H sample times in
// shared memory, then its threads run over (point, bin) pairs, bins fastest,
// so each warp touches contiguous accumulators.  The terms go into the FP32
// partial sums; every kFaceChunk-th call of the run (by the step counter)
// adds those into the FP64 sums and clears them.
__global__ void __launch_bounds__(256) k_face_dft(DevFaceProbes fp, DevFields f, DevGrid g,
                                                  const long long* step_ctr, double dt) {
    const long long n1 = step_ctr[0];         // n + 1
    if (n1 % fp.every != 0) return;
    const bool flush = (n1 / fp.every) % kFaceChunk == kFaceChunk - 1;
    extern __shared__ float2 ph[];            // [0, K): E times, [K, 2K): H times
    const int face = blockIdx.y;
    const int axis = face >> 1;
    const int np = fp.npts[face];
    const int p0 = blockIdx.x * fp.pts_per_block;
    if (p0 >= np) return;
    const int p1 = min(np, p0 + fp.pts_per_block);
    const int plane = fp.plane[face];
    const int K = fp.nfreq;
    const int na = fp.na[face];
    const double tE = (double)n1 * dt, tH = tE - 0.5 * dt;
    for (int q = threadIdx.x; q < 2 * K; q += blockDim.x)
        ph[q] = phase_f32(fp.omega[q % K], q < K ? tE : tH);
    __syncthreads();
    const int work = K * (p1 - p0);
    for (int q = threadIdx.x; q < work; q += blockDim.x) {
        const int kk = q % K, p = p0 + q / K;
        const float2 wE = ph[kk], wH = ph[K + kk];
        const int ia = p % na, ib = p / na;
        // transverse coordinates of point (ia, ib): (a, b) axes per face
        const int ca = fp.r0a[face] + ia * fp.stride, cb = fp.r0b[face] + ib * fp.stride;
        float Ea = 0.f, Eb = 0.f, Ha = 0.f, Hb = 0.f;
        if (axis == 0) {        // x-face: points (j = ca, k = cb); (a, b) = (y, z)
            if (plane < g.nx) {
                const int64_t c = plane + (int64_t)g.nx * ca + g.nxy * cb;
                Ea = f.ey[c]; Eb = f.ez[c];
            }
            if (plane >= 1) {
                const int64_t c = (plane - 1) + (int64_t)g.nx * ca + g.nxy * cb;
                Ha = f.hy[c]; Hb = f.hz[c];
            }
        } else if (axis == 1) { // y-face: points (i = ca, k = cb); fields (z, x)
            if (plane < g.ny) {
                const int64_t c = ca + (int64_t)g.nx * plane + g.nxy * cb;
                Ea = f.ez[c]; Eb = f.ex[c];
            }
            if (plane >= 1) {
                const int64_t c = ca + (int64_t)g.nx * (plane - 1) + g.nxy * cb;
                Ha = f.hz[c]; Hb = f.hx[c];
            }
        } else {                // z-face: points (i = ca, j = cb); (a, b) = (x, y)
            if (plane < g.nz) {
                const int64_t c = ca + (int64_t)g.nx * cb + g.nxy * plane;
                Ea = f.ex[c]; Eb = f.ey[c];
            }
            if (plane >= 1) {
                const int64_t c = ca + (int64_t)g.nx * cb + g.nxy * (plane - 1);
                Ha = f.hx[c]; Hb = f.hy[c];
            }
        }
        const int64_t at = (((int64_t)fp.offset[face] + p) * 4) * K + kk;
        float2* a32 = fp.acc32 + at;
        float2 v[4] = {a32[0], a32[K], a32[2 * K], a32[3 * K]};
        const float val[4] = {Ea, Eb, Ha, Hb};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float2 w = r < 2 ? wE : wH;
            v[r].x = fmaf(val[r], w.x, v[r].x);
            v[r].y = fmaf(val[r], w.y, v[r].y);
        }
        if (flush) {
            double2* a = fp.acc + at;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                double2 d = a[r * K];
                d.x += (double)v[r].x;
                d.y += (double)v[r].y;
                a[r * K] = d;
                v[r] = make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) a32[r * K] = v[r];
    }
}

// Energy, pass 1: per-block partial sums of eps_r |E_s|^2 + |H_s|^2 (FP64)
// into `partial` (one double per block), non-finite values flagged.
__global__ void __launch_bounds__(256) k_energy_partial(DevFields f, int64_t ncell,
                                                        const float* lut_eps, double* partial,
                                                        int* nonfinite) {
    double acc = 0.0;
    bool bad = false;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
         c += (int64_t)gridDim.x * blockDim.x) {
        const float e2 = f.ex[c] * f.ex[c] + f.ey[c] * f.ey[c] + f.ez[c] * f.ez[c];
        const float h2 = f.hx[c] * f.hx[c] + f.hy[c] * f.hy[c] + f.hz[c] * f.hz[c];
        const double eps = f.inv_eps ? 1.0 / (double)f.inv_eps[c] : (double)lut_eps[f.mat[c] & 0x7f];
        const double v = eps * (double)e2 + (double)h2;
        bad |= !isfinite(e2) || !isfinite(h2);
        acc += v;
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) partial[blockIdx.x] = acc;
    }
    if (bad) atomicOr(nonfinite, 1);
}

// Energy, pass 2: one block sums the partials in a fixed order.
__global__ void k_energy_final(const double* partial, int nparts, double* out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) acc += partial[q];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        acc = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) *out = acc;
    }
}

// Philox on n counters (diagnostic entry point).
__global__ void k_philox(const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = philox4x32_10(ctr[t], k0, k1);
}

// ------------------------------------------------------------------ launchers

void launch_philox(const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, int n, cudaStream_t s) {
    k_philox<<<(n + 255) / 256, 256, 0, s>>>(ctr, k0, k1, out, n);
}

void launch_point_dft(const DevPointProbes& pp, const DevFields& f, const long long* ctr,
                      double dt, cudaStream_t s) {
    if (pp.count <= 0) return;
    k_point_dft<<<dim3(pp.count, (pp.nfreq + 31) / 32, 1), 32, 0, s>>>(pp, f.ex, f.ey, f.ez, ctr, dt);
}

void launch_face_dft(const DevFaceProbes& fp, const DevFields& f, const DevGrid& g,
                     const long long* ctr, double dt, cudaStream_t s) {
    if (!fp.on) return;
    int maxpts = 0;
    for (int q = 0; q < 6; ++q) maxpts = fp.npts[q] > maxpts ? fp.npts[q] : maxpts;
    if (maxpts == 0) return;
    dim3 grid((maxpts + fp.pts_per_block - 1) / fp.pts_per_block, 6);
    const size_t smem = sizeof(float2) * 2 * (size_t)fp.nfreq;
    static size_t attr_set = 48 * 1024;   // largest dynamic shared memory allowed so far
    if (smem > attr_set) {
        cudaFuncSetAttribute(k_face_dft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set = smem;
    }
    k_face_dft<<<grid, 256, smem, s>>>(fp, f, g, ctr, dt);
}

// Plane DFT: one thread per plane cell; the block forms the phase factors
// exp(i w_k t_{n+1}) once in shared memory.
__global__ void k_plane_dft(DevPlaneProbe pp, DevFields f, DevGrid g, const long long* step_ctr,
                            double dt) {
    const long long n1 = step_ctr[0];         // n + 1
    if (n1 % pp.every != 0) return;
    __shared__ double2 ph[kPlaneMaxFreq];
    const double t = (double)n1 * dt;
    for (int kk = threadIdx.x; kk < pp.nfreq; kk += blockDim.x) {
        const float2 w = phase_f32(pp.omega[kk], t);
        ph[kk] = make_double2(w.x, w.y);
    }
    __syncthreads();
    const uint32_t nxy = g.nxy;
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nxy) return;
    const uint32_t c = p + nxy * (uint32_t)pp.k;
    const double e[3] = {(double)f.ex[c], (double)f.ey[c], (double)f.ez[c]};
    for (int kk = 0; kk < pp.nfreq; ++kk) {
        const double2 w = ph[kk];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            double2* a = pp.acc + ((size_t)kk * 3 + q) * nxy + p;
            double2 v = *a;
            v.x += e[q] * w.x;
            v.y += e[q] * w.y;
            *a = v;
        }
    }
}

// Energy density of plane z = k: (eps_r |E|^2 + |H|^2) / 2 in units of eps0 E0^2.
__global__ void k_plane_energy(DevFields f, DevGrid g, int k, const float* lut_eps, double* out) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.nxy) return;
    const uint32_t c = p + g.nxy * (uint32_t)k;
    const double eps = f.inv_eps ? 1.0 / (double)f.inv_eps[c] : (double)lut_eps[f.mat[c] & 0x7f];
    const double ex = f.ex[c], ey = f.ey[c], ez = f.ez[c];
    const double hx = f.hx[c], hy = f.hy[c], hz = f.hz[c];
    out[p] = 0.5 * (eps * (ex * ex + ey * ey + ez * ez) + (hx * hx + hy * hy + hz * hz));
}

void launch_plane_dft(const DevPlaneProbe& pp, const DevFields& f, const DevGrid& g,
                      const long long* ctr, double dt, cudaStream_t s) {
    const unsigned blocks = (g.nxy + 255) / 256;
    k_plane_dft<<<blocks, 256, 0, s>>>(pp, f, g, ctr, dt);
}

void launch_plane_energy(const DevFields& f, const DevGrid& g, int k, const float* lut_eps,
                         double* out, cudaStream_t s) {
    const unsigned blocks = (g.nxy + 255) / 256;
    k_plane_energy<<<blocks, 256, 0, s>>>(f, g, k, lut_eps, out);
}

__global__ void k_flux_sum(const double* slots, double* out, double scale) {
    const int q = threadIdx.x;
    if (q >= 6) return;
    double v = 0.0;
    for (int t = 0; t < kFluxSlots; ++t) v += slots[q * kFluxSlots + t];
    out[q] = v * scale;
}

// ------------------------------------------------------------ gain-cell list
// Three passes over chunks of kGainChunk cells: the gain cells of each chunk
// counted, the counts turned into each chunk's first list position (one
// block, in order), then each chunk's gain cells written in increasing
// order.  A block of kGainThreads threads takes one chunk, each thread 16
// consecutive material bytes (one uint4; a chunk starts 16-byte aligned); in
// the scatter a block-wide prefix sum of the threads' counts places every
// gain cell after those before it in shared memory, and the chunk's list is
// then copied out whole (coalesced stores).
constexpr int kGainVec = 16;   // material bytes per thread
constexpr int kGainThreads = 512;
constexpr int kGainChunk = kGainVec * kGainThreads;

// Bit 7 of each of the 16 bytes in v (the gain flag): bit e of the result
// for byte e.
__device__ __forceinline__ unsigned gain_bits16(uint4 v) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    unsigned m = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t g = (w[q] >> 7) & 0x01010101u;   // byte e -> bit 8 e
        m |= ((g | (g >> 7) | (g >> 14) | (g >> 21)) & 0xfu) << (4 * q);
    }
    return m;
}

// The gain bits of the 16 cells [c, c + 16) (cells at or past c1 read as
// not gain).
__device__ __forceinline__ unsigned gain_bits_at(const uint8_t* mat, int64_t c, int64_t c1) {
    if (c + kGainVec <= c1) return gain_bits16(*reinterpret_cast<const uint4*>(mat + c));
    unsigned m = 0;
    for (int e = 0; e < kGainVec && c + e < c1; ++e) m |= (unsigned)(mat[c + e] >> 7) << e;
    return m;
}

__global__ void __launch_bounds__(kGainThreads) k_gain_count(const uint8_t* mat, int64_t N, uint32_t* counts) {
    __shared__ uint32_t wsum[32];
    const int64_t c0 = (int64_t)blockIdx.x * kGainChunk;
    const int64_t c1 = min(N, c0 + kGainChunk);
    uint32_t n = 0;
    for (int64_t c = c0 + (int64_t)kGainVec * threadIdx.x; c < c1; c += (int64_t)kGainVec * blockDim.x)
        n += __popc(gain_bits_at(mat, c, c1));
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
        counts[blockIdx.x] = t;
    }
}

// counts[0, nchunks) -> exclusive prefix sums, in place (one block).
__global__ void __launch_bounds__(1024) k_gain_scan(uint32_t* counts, int nchunks) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int base = 0; base < nchunks; base += blockDim.x) {
        const int q = base + threadIdx.x;
        const uint32_t v = q < nchunks ? counts[q] : 0u;
        uint32_t x = v;   // inclusive scan within the warp
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t z = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
                if (lane >= o) z += y;
            }
            wsum[lane] = z;   // inclusive prefix of the warp totals
        }
        __syncthreads();
        const uint32_t before = carry + (warp > 0 ? wsum[warp - 1] : 0u) + (x - v);
        if (q < nchunks) counts[q] = before;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += wsum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kGainThreads) k_gain_scatter(const uint8_t* mat, int64_t N,
                                                               const uint32_t* first, uint32_t* list) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t cells[kGainChunk];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t c0 = (int64_t)blockIdx.x * kGainChunk;
    const int64_t c1 = min(N, c0 + kGainChunk);
    const int64_t c = c0 + (int64_t)kGainVec * threadIdx.x;
    unsigned m = c < c1 ? gain_bits_at(mat, c, c1) : 0u;
    const uint32_t cnt = __popc(m);
    uint32_t x = cnt;   // inclusive scan of the counts within the warp
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t z = lane < nw ? wsum[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        wsum[lane] = z;   // inclusive prefix of the warp totals
    }
    __syncthreads();
    uint32_t at = (warp > 0 ? wsum[warp - 1] : 0u) + (x - cnt);
    while (m) {
        const int e = __ffs(m) - 1;
        m &= m - 1;
        cells[at++] = (uint32_t)(c + e);
    }
    __syncthreads();
    const uint32_t total = wsum[nw - 1], pos = first[blockIdx.x];
    for (uint32_t q = threadIdx.x; q < total; q += blockDim.x) list[pos + q] = cells[q];
}

// counts[nchunks] = the total (after the scan: the last chunk's first
// position plus its count, kept aside before the scan overwrites it).
__global__ void k_gain_total(uint32_t* counts, int nchunks) {
    if (threadIdx.x == 0) counts[nchunks + 1] = counts[nchunks - 1];
}
__global__ void k_gain_total2(uint32_t* counts, int nchunks) {
    if (threadIdx.x == 0) counts[nchunks] = counts[nchunks - 1] + counts[nchunks + 1];
}

static int gain_chunks(int64_t N) { return (int)((N + kGainChunk - 1) / kGainChunk); }

size_t gain_list_scratch(int64_t N) { return (size_t)gain_chunks(N) + 2; }

void launch_gain_count(const uint8_t* mat, int64_t N, uint32_t* scratch, cudaStream_t s) {
    const int nchunks = gain_chunks(N);
    if (nchunks == 0) return;
    k_gain_count<<<nchunks, kGainThreads, 0, s>>>(mat, N, scratch);
    k_gain_total<<<1, 32, 0, s>>>(scratch, nchunks);
    k_gain_scan<<<1, 1024, 0, s>>>(scratch, nchunks);
    k_gain_total2<<<1, 32, 0, s>>>(scratch, nchunks);
}

void launch_gain_scatter(const uint8_t* mat, int64_t N, const uint32_t* scratch, uint32_t* list,
                         cudaStream_t s) {
    const int nchunks = gain_chunks(N);
    if (nchunks == 0) return;
    k_gain_scatter<<<nchunks, kGainThreads, 0, s>>>(mat, N, scratch, list);
}

// ------------------------------------------------------------ material map
// The eps_r map's distinct values (bit patterns) into a table of kMatKeys
// entries by compare-and-swap on the first free slot, so the table fills as
// a prefix, with the first cell holding each value (atomic minimum);
// flags[0] is set by a value not finite or below 1, flags[1] by a value that
// finds the table full.  Each warp walks its own contiguous stretch of the
// map 128 cells at a time (four coalesced loads issued together, then taken
// 32 cells at a time in cell order); of the lanes holding one value only the
// lowest (the value's lowest cell of those 32) goes to the table, and only
// for a value the warp has not recorded yet (a short list of the warp's
// values, the same in every lane), so the table sees a few requests per warp.
constexpr int kWarpSeen = 8;
constexpr int kKeysUnroll = 4;

__device__ __forceinline__ bool eps_bits_valid(uint32_t b) {
    return (b - 0x3f800000u) < 0x40000000u;   // 1 <= eps_r < inf, sign clear
}

__global__ void __launch_bounds__(256) k_mat_keys(const float* eps, int64_t N, uint32_t* keys,
                                                  uint32_t* first, int* flags) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    constexpr int kStep = 32 * kKeysUnroll;
    const int64_t span = ((N + nwarps - 1) / nwarps + kStep - 1) / kStep * kStep;
    const int64_t c0 = w * span, c1 = min(N, c0 + span);
    uint32_t seen[kWarpSeen];
    int nseen = 0;
    for (int64_t base = c0; base < c1; base += kStep) {
        uint32_t bv[kKeysUnroll];
#pragma unroll
        for (int u = 0; u < kKeysUnroll; ++u) {
            const int64_t c = base + 32 * u + lane;
            bv[u] = c < c1 ? __float_as_uint(__ldcs(eps + c)) : kNoKey;
        }
#pragma unroll
        for (int u = 0; u < kKeysUnroll; ++u) {
            const int64_t c = base + 32 * u + lane;
            const bool in = c < c1;
            const uint32_t b = bv[u];
            const bool ok = !in || eps_bits_valid(b);
            if (!ok) flags[0] = 1;
            const uint32_t bb = ok ? b : kNoKey;   // invalid and absent lanes take no part
            // 32 cells of one value the warp has recorded already (the
            // inside of a sphere or a void): nothing to do
            const uint32_t b0 = __shfl_sync(full, bb, 0);
            if (__all_sync(full, bb == b0)) {
                bool have = b0 == kNoKey;
                for (int q = 0; q < nseen; ++q) have |= seen[q] == b0;
                if (have) continue;
            }
            const unsigned same = __match_any_sync(full, bb);
            const bool leader = bb != kNoKey && lane == __ffs(same) - 1;
            bool known = false;
            for (int q = 0; q < nseen; ++q) known |= seen[q] == bb;
            const bool ask = leader && !known;
            if (ask) {
                int at = -1;
                for (int q = 0; q < kMatKeys && at < 0; ++q) {
                    uint32_t k = *reinterpret_cast<volatile uint32_t*>(keys + q);
                    if (k == kNoKey) {
                        const uint32_t old = atomicCAS(keys + q, kNoKey, bb);
                        k = old == kNoKey ? bb : old;
                    }
                    if (k == bb) at = q;
                }
                if (at < 0) flags[1] = 1;
                else atomicMin(first + at, (uint32_t)c);
            }
            // the values just recorded join the warp's list (in every lane)
            unsigned fresh = __ballot_sync(full, ask);
            while (fresh) {
                const int src = __ffs(fresh) - 1;
                fresh &= fresh - 1;
                const uint32_t v = __shfl_sync(full, bb, src);
                if (nseen < kWarpSeen) seen[nseen++] = v;
            }
        }
    }
}

// The material byte of one cell from the (sorted) table: its id in keys[0,
// n) (0 for a dense map, whose 1/eps_r goes per cell into inv_eps) and bit 7
// for a gain cell; last / last_id remember the previous lookup (runs of one
// value skip the table search).
__device__ __forceinline__ uint8_t mat_byte(float v, uint8_t g, const uint32_t* sk, int n, int dense,
                                            int gain_on, uint32_t& last, uint8_t& last_id) {
    uint8_t id = 0;
    if (!dense) {
        const uint32_t b = __float_as_uint(v);
        if (b == last) {
            id = last_id;
        } else {
            for (int q = 0; q < n; ++q)
                if (sk[q] == b) {
                    id = (uint8_t)q;
                    break;
                }
            last = b;
            last_id = id;
        }
    }
    return (uint8_t)(id | ((gain_on && g != 0) ? 0x80 : 0x00));
}

// The material bytes of the map, four cells per thread and pass (the eps_r
// map, the gain mask and the material bytes start 16- / 4-byte aligned; the
// last N % 4 cells one at a time).
__global__ void __launch_bounds__(256) k_mat_ids(const float* eps, const uint8_t* gain, int64_t N,
                                                 const uint32_t* keys, int n, int dense, int gain_on,
                                                 uint8_t* mat, float* inv_eps) {
    __shared__ uint32_t sk[kMatKeys];
    for (int q = threadIdx.x; q < kMatKeys; q += blockDim.x) sk[q] = q < n ? keys[q] : kNoKey;
    __syncthreads();
    uint32_t last = kNoKey;
    uint8_t last_id = 0;
    const int64_t n4 = N / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n4; t += stride) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(eps) + t);
        const uchar4 g = __ldcs(reinterpret_cast<const uchar4*>(gain) + t);
        if (dense)
            reinterpret_cast<float4*>(inv_eps)[t] =
                make_float4((float)(1.0 / (double)v.x), (float)(1.0 / (double)v.y),
                            (float)(1.0 / (double)v.z), (float)(1.0 / (double)v.w));
        uchar4 m;
        m.x = mat_byte(v.x, g.x, sk, n, dense, gain_on, last, last_id);
        m.y = mat_byte(v.y, g.y, sk, n, dense, gain_on, last, last_id);
        m.z = mat_byte(v.z, g.z, sk, n, dense, gain_on, last, last_id);
        m.w = mat_byte(v.w, g.w, sk, n, dense, gain_on, last, last_id);
        reinterpret_cast<uchar4*>(mat)[t] = m;
    }
    for (int64_t c = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < N; c += stride) {
        const float v = eps[c];
        if (dense) inv_eps[c] = (float)(1.0 / (double)v);
        mat[c] = mat_byte(v, gain[c], sk, n, dense, gain_on, last, last_id);
    }
}

void launch_mat_keys(const float* eps, int64_t N, uint32_t* keys, uint32_t* first, int* flags,
                     cudaStream_t s) {
    k_mat_keys<<<1216, 256, 0, s>>>(eps, N, keys, first, flags);
}

void launch_mat_ids(const float* eps, const uint8_t* gain, int64_t N, const uint32_t* keys, int n,
                    bool dense, bool gain_on, uint8_t* mat, float* inv_eps, cudaStream_t s) {
    k_mat_ids<<<1216, 256, 0, s>>>(eps, gain, N, keys, n, dense ? 1 : 0, gain_on ? 1 : 0, mat, inv_eps);
}

void launch_flux_sum(const double* slots, double* out, double scale, cudaStream_t s) {
    k_flux_sum<<<1, 32, 0, s>>>(slots, out, scale);
}

void launch_energy(const DevFields& f, int64_t ncell, const float* lut_eps, double* partial,
                   int nparts, int* nonfinite, double* out, cudaStream_t s) {
    k_energy_partial<<<nparts, 256, 0, s>>>(f, ncell, lut_eps, partial, nonfinite);
    k_energy_final<<<1, 1024, 0, s>>>(partial, nparts, out);
}

}  // namespace mb
