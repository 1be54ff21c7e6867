// Boundary planes of z-slab contexts: one grid split along z into slabs,
// each advanced by its own context, exchanges one plane per neighbour per
// step (the paper's "Simulations" paragraph runs its grid distributed over
// 256 processors; here the slabs may sit on one GPU or on several).
//
// A slab context holds its own planes plus a ghost plane next to each
// neighbour.  Before every step, each ghost plane receives the whole state
// of the neighbour's boundary plane at time n (E^n, H^{n-1/2}, P, J, the
// populations and the x / y CPML memories; the cut planes lie outside the
// z-CPML).  The slab's ordinary step then computes every own cell exactly as
// the whole grid does: the E update of the lowest own plane reads H^{n+1/2}
// of the ghost below, which the step recomputes there from the same inputs
// as the neighbour; the H update of the highest own plane reads E^n of the
// ghost above.  What the step writes into ghost planes is never read by an
// own cell before the next exchange overwrites it.
#include "mb_ctx.h"

namespace {

// One plane of a context's state, at local plane k of the current copy.
struct HaloPlane {
    float* eh;       // E, H of the current copy (6 arrays of N floats)
    float* fields;   // the context's 15 arrays (P, J, n1..n3 from array 6)
    float* psx;      // x-slab CPML memories of the current copy (or null)
    float* psy;      // y-slab CPML memories of the current copy (or null)
    int64_t N;
    int64_t nxy;
    int nx, ny, nz, L2;
    int k;
};

// Floats of one packed plane: the 15 arrays (nx ny each), then the x-slab
// memories (4 planes f of ny 2L), then the y-slab memories (4 planes f of
// 2L nx).
int64_t halo_floats(const mb_ctx* c) {
    const int64_t L2 = 2 * (int64_t)c->p.npml;
    return 15 * (int64_t)c->nx * c->ny + 4 * (int64_t)c->ny * L2 + 4 * L2 * c->nx;
}

// Address of float q of the packed plane in the context's arrays (the
// x-slab memory of (f, k, j, s) sits at ((f nz + k) ny + j) 2L + s, the
// y-slab memory of (f, k, s, i) at ((f nz + k) 2L + s) nx + i).
__device__ __forceinline__ float* halo_addr(const HaloPlane& h, int64_t q) {
    const int64_t a = 15 * h.nxy;
    if (q < a) {
        const int64_t seg = q / h.nxy;
        const int64_t r = q - seg * h.nxy;
        float* base = (seg < 6 ? h.eh : h.fields) + seg * h.N;
        return base + (int64_t)h.k * h.nxy + r;
    }
    q -= a;
    const int64_t bx = (int64_t)h.ny * h.L2;
    if (q < 4 * bx) {
        const int64_t f = q / bx;
        return h.psx + (f * h.nz + h.k) * bx + (q - f * bx);
    }
    q -= 4 * bx;
    const int64_t by = (int64_t)h.L2 * h.nx;
    const int64_t f = q / by;
    return h.psy + (f * h.nz + h.k) * by + (q - f * by);
}

template <bool PACK>
__global__ void k_halo(HaloPlane h, float* buf, int64_t total) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        float* p = halo_addr(h, q);
        if (PACK) buf[q] = *p;
        else *p = buf[q];
    }
}

int halo_launch(mb_ctx* c, int k, float* buf, bool pack) {
    HaloPlane h;
    h.eh = mbi::eh_of(c, c->parity);
    h.fields = c->d_fields;
    h.psx = mbi::psi_of(c, c->parity, 0);
    h.psy = mbi::psi_of(c, c->parity, 1);
    h.N = c->ncell;
    h.nxy = (int64_t)c->nx * c->ny;
    h.nx = c->nx;
    h.ny = c->ny;
    h.nz = c->nz;
    h.L2 = 2 * c->p.npml;
    h.k = k;
    const int64_t total = halo_floats(c);
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((total + threads - 1) / threads, 152 * 8);
    if (pack) k_halo<true><<<blocks, threads, 0, c->stream>>>(h, buf, total);
    else k_halo<false><<<blocks, threads, 0, c->stream>>>(h, buf, total);
    MB_CUDA(c, cudaGetLastError());
    c->launches += 1;
    return MB_OK;
}

}  // namespace

extern "C" int mb_halo_bytes(mb_ctx* c, size_t* bytes) {
    if (int rc = mbi::check_ctx_nojoin(c)) return rc;
    if (!bytes) return mbi::fail(c, MB_ERR_ARG, "null output");
    *bytes = sizeof(float) * (size_t)halo_floats(c);
    return MB_OK;
}

extern "C" int mb_halo_pack(mb_ctx* c, int side, void* d_buf) {
    if (int rc = mbi::check_ctx(c)) return rc;
    if (!c->slab) return mbi::fail(c, MB_ERR_STATE, "not a z-slab context");
    if ((side != 0 && side != 1) || !d_buf) return mbi::fail(c, MB_ERR_ARG, "side must be 0 or 1, buffer non-null");
    return halo_launch(c, side ? c->own_hi - 1 : c->own_lo, static_cast<float*>(d_buf), true);
}

extern "C" int mb_halo_unpack(mb_ctx* c, int side, const void* d_buf) {
    if (int rc = mbi::check_ctx(c)) return rc;
    if (!c->slab) return mbi::fail(c, MB_ERR_STATE, "not a z-slab context");
    if ((side != 0 && side != 1) || !d_buf) return mbi::fail(c, MB_ERR_ARG, "side must be 0 or 1, buffer non-null");
    if (side == 0 && c->own_lo != 1) return mbi::fail(c, MB_ERR_STATE, "no ghost plane below (the slab starts the grid)");
    if (side == 1 && c->own_hi != c->nz - 1) return mbi::fail(c, MB_ERR_STATE, "no ghost plane above (the slab ends the grid)");
    return halo_launch(c, side ? c->nz - 1 : 0, const_cast<float*>(static_cast<const float*>(d_buf)), false);
}
