// Bound states of the dimensionless spectral-envelope equation of the
// random-laser theory (the paper's Eq. g5, "Gross-Pitaevskii equation"
// paragraph):
//     -phi'' + tau^2 phi + phi^3 = E phi,   phi > 0,  phi(+-L) = 0,
// for a batch of eigenvalues E > 1, and the spectral waist and peak of each
// (Figs. 3, 5).  Second-order differences on tau_i = -L + i h (i = 1..n,
// h = 2L/(n+1)), Newton's method with a tridiagonal (Thomas) solve per
// iteration, all in FP64; one thread per eigenvalue, its arrays in global
// scratch interleaved across the eigenvalues (element i of eigenvalue q at
// i nE + q), so that the threads of a warp touch consecutive addresses.  Newton starts from the larger of the Thomas-Fermi profile
// sqrt(max(E - tau^2, 0)) and the first-order solution near threshold
// 2^{1/4} sqrt(E - 1) exp(-tau^2 / 2) and stops when the residual is below
// 1e-12 max(1, E) or the step stagnates at rounding level; a result whose
// residual stays above 1e-9 max(1, E), or that collapses towards the trivial
// solution phi = 0, is reported as not converged.
#include "mb_host.h"

#include <cmath>
#include <string>
#include <vector>

namespace {

constexpr int kGpMaxIter = 100;

// A thread's array with its elements nE apart (the interleaved layout).
struct Strided {
    double* p;
    size_t s;
    __device__ double& operator[](int i) const { return p[(size_t)i * s]; }
};

__device__ double gp_residual(const Strided& phi, int i, int n, double t2, double ih2, double E) {
    const double l = i > 0 ? phi[i - 1] : 0.0;
    const double r = i < n - 1 ? phi[i + 1] : 0.0;
    const double p = phi[i];
    return -(l - 2.0 * p + r) * ih2 + t2 * p + p * p * p - E * p;
}

// One thread per eigenvalue: phi (n), and the Thomas sweep's scratch (2n),
// all interleaved across the eigenvalues.
__global__ void k_gp_solve(const double* Es, int nE, int n, double* phi_all, double* scratch,
                           double* w_out, double* p_out, int* status) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nE) return;
    const double E = Es[q];
    const Strided phi{phi_all + q, (size_t)nE};
    const Strided cp{scratch + q, (size_t)nE};
    const Strided dp{scratch + (size_t)n * nE + q, (size_t)nE};
    const double L = sqrt(E) + 8.0;
    const double h = 2.0 * L / (n + 1);
    const double ih2 = 1.0 / (h * h);
    const double amp = pow(2.0, 0.25) * sqrt(E - 1.0);
    for (int i = 0; i < n; ++i) {
        const double t = -L + h * (i + 1);
        const double tf = sqrt(fmax(E - t * t, 0.0));
        const double g = amp * exp(-0.5 * t * t);
        phi[i] = fmax(tf, g);
    }
    const double tol = 1e-12 * fmax(1.0, E);
    int ok = 0;
    for (int it = 0; it < kGpMaxIter; ++it) {
        // residual into dp, its sup norm
        double rmax = 0.0;
        for (int i = 0; i < n; ++i) {
            const double t = -L + h * (i + 1);
            const double f = gp_residual(phi, i, n, t * t, ih2, E);
            dp[i] = f;
            rmax = fmax(rmax, fabs(f));
        }
        if (rmax < tol) {
            ok = 1;
            break;
        }
        // Thomas: (-ih2) x_{i-1} + (2 ih2 + tau^2 + 3 phi^2 - E) x_i + (-ih2) x_{i+1} = f_i
        const double off = -ih2;
        double t0 = -L + h;
        double b = 2.0 * ih2 + t0 * t0 + 3.0 * phi[0] * phi[0] - E;
        cp[0] = off / b;
        dp[0] = dp[0] / b;
        for (int i = 1; i < n; ++i) {
            const double t = -L + h * (i + 1);
            const double bi = 2.0 * ih2 + t * t + 3.0 * phi[i] * phi[i] - E;
            const double m = bi - off * cp[i - 1];
            cp[i] = i < n - 1 ? off / m : 0.0;
            dp[i] = (dp[i] - off * dp[i - 1]) / m;
        }
        double x = dp[n - 1];
        double dmax = fabs(x), pmx = 0.0;
        phi[n - 1] -= x;
        for (int i = n - 2; i >= 0; --i) {
            x = dp[i] - cp[i] * x;
            phi[i] -= x;
            dmax = fmax(dmax, fabs(x));
            pmx = fmax(pmx, phi[i]);
        }
        if (dmax <= 1e-14 * fmax(1.0, pmx)) break;   // stagnated at rounding level
    }
    if (!ok) {
        // the residual's rounding floor (~1/h^2 times eps) can lie above tol:
        // once the steps stagnate, accept a residual below 1e-9 max(1, E)
        double rmax = 0.0;
        for (int i = 0; i < n; ++i) {
            const double t = -L + h * (i + 1);
            rmax = fmax(rmax, fabs(gp_residual(phi, i, n, t * t, ih2, E)));
        }
        ok = rmax < 1e-9 * fmax(1.0, E);
    }
    // features: p = (h sum phi)^2 / (4 pi^2); w = sqrt(sum dphi^2 / sum phi^2) / (2 pi)
    double s1 = 0.0, s2 = 0.0, sd = 0.0, pmax = 0.0, prev = 0.0;
    for (int i = 0; i < n; ++i) {
        const double p = phi[i];
        s1 += p;
        s2 += p * p;
        sd += (p - prev) * (p - prev);
        prev = p;
        pmax = fmax(pmax, p);
    }
    sd += prev * prev;   // the step to phi(L) = 0
    const double pi = 3.14159265358979323846;
    const double hs1 = h * s1;
    p_out[q] = hs1 * hs1 / (4.0 * pi * pi);
    w_out[q] = sqrt((sd / (h * h)) / s2) / (2.0 * pi);
    if (ok && pmax < 0.5 * amp) ok = 0;   // collapsed towards phi = 0
    status[q] = ok;
}

}  // namespace

extern "C" int mb_gp_features(const double* E, int nE, int n_grid, double* w_phi, double* p_phi,
                              double* phi_out) {
    if (!E || nE < 1 || n_grid < 16 || n_grid > (1 << 20) || !w_phi || !p_phi) {
        mb::set_thread_error("bad arguments: nE >= 1, 16 <= n_grid <= 2^20, outputs non-null");
        return MB_ERR_ARG;
    }
    for (int q = 0; q < nE; ++q)
        if (!(E[q] > 1.0) || !std::isfinite(E[q])) {
            mb::set_thread_error("every E must be finite and > 1 (bound states exist above threshold)");
            return MB_ERR_ARG;
        }
    const size_t n = (size_t)n_grid;
    double *dE = nullptr, *dphi = nullptr, *dscr = nullptr, *dw = nullptr, *dp = nullptr;
    int* dst = nullptr;
    std::vector<int> st((size_t)nE);
    int rc = MB_OK;
    cudaError_t e = cudaMalloc((void**)&dE, sizeof(double) * nE);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dphi, sizeof(double) * n * nE);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dscr, sizeof(double) * 2 * n * nE);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dw, sizeof(double) * nE);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dp, sizeof(double) * nE);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dst, sizeof(int) * nE);
    if (e == cudaSuccess) e = cudaMemcpy(dE, E, sizeof(double) * nE, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_gp_solve<<<(nE + 63) / 64, 64>>>(dE, nE, n_grid, dphi, dscr, dw, dp, dst);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(w_phi, dw, sizeof(double) * nE, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(p_phi, dp, sizeof(double) * nE, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(st.data(), dst, sizeof(int) * nE, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && phi_out) {
        // device layout [i][q] -> caller's [q][i]
        std::vector<double> t(n * (size_t)nE);
        e = cudaMemcpy(t.data(), dphi, sizeof(double) * n * nE, cudaMemcpyDeviceToHost);
        for (int q = 0; q < nE && e == cudaSuccess; ++q)
            for (size_t i = 0; i < n; ++i) phi_out[(size_t)q * n + i] = t[i * nE + q];
    }
    if (e != cudaSuccess) {
        mb::set_thread_error(std::string("gp solve: ") + cudaGetErrorString(e));
        rc = e == cudaErrorMemoryAllocation ? MB_ERR_OOM : MB_ERR_CUDA;
    } else {
        for (int q = 0; q < nE; ++q)
            if (!st[q]) {
                mb::set_thread_error("Newton did not converge to a bound state for E = " + std::to_string(E[q]));
                rc = MB_ERR_STATE;
                break;
            }
    }
    void* bufs[] = {dE, dphi, dscr, dw, dp, dst};
    for (void* b : bufs)
        if (b) cudaFree(b);
    return rc;
}
