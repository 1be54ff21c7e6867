/*
 * mb_fdtd.h — C ABI of the GB300 Maxwell–Bloch FDTD step.
 *
 * The operation: one time step of the vectorial Maxwell–Bloch (MB) random-
 * laser model of Conti, Leonetti, Fratalocchi, Angelani, Ruocco,
 * "Condensation in disordered lasers: theory, 3D+1 simulations and
 * experiments" (arXiv:0809.1547), section "Simulations": an FDTD (Yee grid)
 * solution of Maxwell's equations through a packing of TiO2 spheres (n=2.9)
 * whose voids hold a four-level gain medium (lambda0 = 590 nm, 230 nm gain
 * bandwidth ~ 1/t_g) pumped at a constant rate, with spontaneous emission
 * as a stochastic (Langevin) term.  The paper prints no equations; the scheme
 * implemented is the standard four-level Lorentz-oscillator MB-FDTD model:
 *
 *   H^{n+1/2} = H^{n-1/2} - dt/mu0 curl E^n                 (+ CPML)
 *   J^{n+1/2} = [(1-a) J^{n-1/2} + dt (xi (N1-N2) E^n - w0^2 P^n + F^n)]/(1+a)
 *   P^{n+1}   = P^n + dt J^{n+1/2}                           (gain cells)
 *   E^{n+1}   = E^n + dt/(eps0 eps_r) (curl H^{n+1/2} - J^{n+1/2} - J_src)
 *   N^{n+1}   = M N^n + m (E^n+E^{n+1})/2 . J^{n+1/2} / (hbar w0)
 *
 * with a = dw_a dt/2, M, m the Crank–Nicolson propagator of the four-level
 * rate equations (pump W_p from N0 to N3), and F a Langevin force drawn from
 * Philox4x32-10 keyed by (seed, cell, step).  PEC walls bound the grid, a
 * CPML of npml cells lines every face.
 *
 * Conventions.  Grid n_x x n_y x n_z, x fastest: cell index
 * c = i + n_x (j + n_y k).  Cell (i,j,k) owns Ex(i+1/2,j,k), Ey(i,j+1/2,k),
 * Ez(i,j,k+1/2), Hx(i,j+1/2,k+1/2), Hy(i+1/2,j,k+1/2), Hz(i+1/2,j+1/2,k),
 * P and J on the E sites and the populations N0..N3.  All host arrays are
 * borrowed and copied during the call; the context owns every device buffer
 * it allocates.  Fields crossing the ABI are in SI units (V/m, A/m, C/m^2,
 * A/m^2, m^-3).  Every call returns MB_OK (0) or a negative MB_ERR_* code and
 * never aborts the process; mb_last_error() then holds a message.  Calls on
 * one context are not thread-safe.  Work is queued on the context's CUDA
 * stream; calls that return host data synchronize that stream.
 */
#ifndef MB_FDTD_H
#define MB_FDTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MB_OK = 0,
    MB_ERR_ARG = -1,        /* bad argument (null pointer, size, index)          */
    MB_ERR_COURANT = -2,    /* dt > dx / (c sqrt 3)                              */
    MB_ERR_OOM = -3,        /* device or host allocation failed                  */
    MB_ERR_MATERIALS = -4,  /* eps_r < 1 or not finite                           */
    MB_ERR_TIMEOUT = -5,    /* a bounded device wait gave up                     */
    MB_ERR_NONFINITE = -6,  /* NaN / Inf found in the fields                     */
    MB_ERR_CUDA = -7,       /* a CUDA runtime call failed                        */
    MB_ERR_STATE = -8       /* call not valid in this state (e.g. no material)  */
};

/* Field identifiers for mb_get_field / mb_set_field. */
enum {
    MB_EX = 0, MB_EY, MB_EZ, MB_HX, MB_HY, MB_HZ,
    MB_PX, MB_PY, MB_PZ, MB_JX, MB_JY, MB_JZ,
    MB_N0, MB_N1, MB_N2, MB_N3,
    MB_NUM_FIELDS
};

/* Physical and numerical parameters (SI).  mb_default_params fills the
 * values of the model: lambda0 = 590 nm and dlambda = 230 nm (paper,
 * "Simulations"); lifetimes tau32 = tau10 = 100 fs, tau21 = 1 ns and the
 * noise amplitude are not given by the paper and are user choices. */
typedef struct mb_params {
    double lambda0;          /* gain centre wavelength (m)                      */
    double dlambda;          /* gain bandwidth (m); dw_a = 2 pi c dlambda/lambda0^2 */
    double tau32, tau21, tau10;  /* level lifetimes (s)                         */
    double a_se;             /* Langevin amplitude (SI); < 0 selects
                                w0 (e dipole_len) sqrt(2 dw_a)                  */
    double dipole_len;       /* dipole length of the default a_se (m)           */
    double n_floor_rel;      /* N_floor / N_a under the noise square root       */
    int    npml;             /* CPML cells per face (>= 0)                      */
    double pml_order;        /* sigma grading exponent                          */
    double pml_sigma_factor; /* sigma_max = factor (order+1) / (eta0 dx)        */
    double pml_alpha_rel;    /* alpha_max = 2 pi eps0 alpha_rel c / lambda0     */
    double n_ref;            /* density (m^-3) fixing the FP32 field scale
                                E0 = sqrt(hbar w0 n_ref / eps0); no effect on
                                the SI results beyond FP32 rounding             */
} mb_params;

typedef struct mb_ctx mb_ctx;

/* Fill *p with the defaults listed above. */
void mb_default_params(mb_params* p);

/* Create a context for one realization on a grid[0] x grid[1] x grid[2] Yee
 * grid with spacing dx (m) and step dt (m, s).  p == NULL selects the
 * defaults.  cuda_stream is a cudaStream_t the context queues its work on
 * (NULL: the context creates its own).  Fields start at zero, eps_r = 1, no
 * gain.  Errors: MB_ERR_ARG (size < 1, dx <= 0), MB_ERR_COURANT, MB_ERR_OOM,
 * MB_ERR_CUDA.  On error *out is NULL. */
int mb_create(mb_ctx** out, const int grid[3], double dx, double dt,
              const mb_params* p, void* cuda_stream);

/* Free every device and host buffer of the context (NULL is accepted). */
int mb_destroy(mb_ctx* ctx);

/* Message of the last failed call on ctx (thread-local text for ctx == NULL). */
const char* mb_last_error(const mb_ctx* ctx);

/* Material: eps_map (host, n cells, x fastest, values >= 1) and gain_mask
 * (host, n cells, nonzero = gain medium, i.e. a void).  The paper's
 * "amplification only in the interstices" is the caller's mask.  N_a is the
 * total atom density (m^-3, N0 = N_a in gain cells at t = 0) and pump the
 * rate W_p (1/s) from N0 to N3, constant in time.  Resets P, J and the
 * populations; fields and probes are kept.  With <= 128 distinct eps values
 * the map is stored as a uint8 material id per cell, otherwise as a dense
 * FP32 1/eps_r map.  Errors: MB_ERR_ARG, MB_ERR_MATERIALS. */
int mb_set_material(mb_ctx* ctx, const float* eps_map, const uint8_t* gain_mask,
                    double N_a, double pump);

/* 64-bit key of the Langevin noise: Philox4x32-10 with key (seed low word,
 * seed high word) and counter (cell index, step, 0, 0). */
int mb_set_seed(mb_ctx* ctx, uint64_t seed);

/* Running-DFT point probe on the three E components of cell ijk:
 * E~_c(w_k) += E_c(t_{n+1}) exp(i w_k t_{n+1}) dt after every step, summed in
 * FP64 on the device (the factor exp(i w t) is formed in FP32 from the angle
 * reduced in FP64), n_freq wavelengths uniformly from lam_min to lam_max.
 * *probe_id receives the probe index.  Errors: MB_ERR_ARG. */
int mb_add_point_probe(mb_ctx* ctx, const int ijk[3], int n_freq,
                       double lam_min, double lam_max, int* probe_id);

/* Face probes on the six faces of the interior box [npml, n - npml)^3: on
 * every stride-th point of each face, the tangential E (on the face plane,
 * at t_{n+1}) and H (half a cell outside, at t_{n+1/2}) are accumulated into
 * running DFTs every `every` steps (1 <= n_freq <= 4096): FP32 sums over 16
 * consecutive accumulations, each added into FP64 sums on the device (the
 * spectrum reads both).  Replaces earlier face probes. */
int mb_add_face_probes(mb_ctx* ctx, int stride, int every, int n_freq,
                       double lam_min, double lam_max);

/* Soft current source J_comp(t) = amp sin(w_s (t - t0)) exp(-((t-t0)/tau)^2)
 * (A/m^2, w_s = 2 pi c / lam) added at cell ijk, component comp (0,1,2), at
 * t = (n + 1/2) dt.  amp = 0 removes the source. */
int mb_set_source(mb_ctx* ctx, const int ijk[3], int comp, double lam,
                  double t0, double tau, double amp);

/* Continuous-wave soft current (the excitation that shows the field of a
 * long-living mode, inset of the paper's Fig. 1 at 586.5 nm):
 * J_comp(t) = amp sin(w_s (t - t0)) (1 - exp(-((t - t0)/tau)^2)) for t >= t0
 * (A/m^2, w_s = 2 pi c / lam; tau is the rise time), at t = (n + 1/2) dt, for
 * the n_steps steps from the first one whose t_{n+1/2} >= t0, zero after.
 * Replaces any source; amp = 0 removes it.  Errors: MB_ERR_ARG (t0 < 0, tau
 * <= 0, 1 <= n_steps <= 2^24 violated, cell outside the grid). */
int mb_set_source_cw(mb_ctx* ctx, const int ijk[3], int comp, double lam, double t0,
                     double tau, double amp, int n_steps);

/* Whole-plane probe on the plane z = k dx (the sample's middle section for
 * k = n_z/2): running FP64 DFTs of Ex, Ey, Ez on every cell of the plane,
 * at t_{n+1}, every `every` steps, n_freq (1..64) wavelengths evenly spaced
 * from lam_min to lam_max.  *probe_id receives its index.  Plane probes are
 * kept by save/load and are not advanced inside a batch.
 * Errors: MB_ERR_ARG, MB_ERR_OOM. */
int mb_add_plane_probe(mb_ctx* ctx, int k, int every, int n_freq, double lam_min,
                       double lam_max, int* probe_id);

/* Mode map of a plane probe at frequency bin `bin`: out_map[i + n_x j] =
 * sum over components of |sum_n E_c(t_n) exp(i w t_n) every dt|^2 in
 * (V s/m)^2 (host array of n_x n_y doubles).  Synchronizes. */
int mb_plane_mode_map(mb_ctx* ctx, int probe_id, int bin, double* out_map);

/* Snapshot of the energy density on the plane z = k dx (the middle-section
 * snapshot of the paper's Fig. 2a): out[i + n_x j] = (eps0 eps_r |E|^2 +
 * mu0 |H|^2)/2 of each cell's own components (J/m^3; the per-cell terms of
 * mb_energy), host array of n_x n_y doubles.  Synchronizes. */
int mb_plane_energy_density(mb_ctx* ctx, int k, double* out);

/* Advance n >= 0 steps (asynchronous on the context's stream; whole chunks
 * of steps replay a captured CUDA graph).  With the single-pass step, the
 * probe DFTs of the steps after the last whole chunk (e.g. every step of
 * mb_step(ctx, 1)) run on the context's second stream beside the next step
 * (they read only the copy that step wrote, which the next step only reads)
 * and may still run when the context's stream passes this call: every later
 * call on the context except mb_step and mb_flux_async first orders the
 * context's stream after them, and mb_join_probes does only that.  The
 * fields, the step count and the face energies are final on the context's
 * stream as usual. */
int mb_step(mb_ctx* ctx, int n);

/* Order the context's stream after the probe launches mb_step left running
 * on the second stream (enqueues event waits; does not block the host): an
 * event the caller records on the context's stream afterwards covers all of
 * the context's work so far.  Errors: MB_ERR_ARG (null context). */
int mb_join_probes(mb_ctx* ctx);

/* Zero the running DFT sums of every probe of the context (point, face and
 * plane probes), on the context's stream after the probe launches still
 * running: the spectra read afterwards cover the steps taken after this call
 * only (a time window of the run; the phases keep the absolute time t_n, so
 * |S|^2 is that of the window's samples).  The face energies (mb_energy's
 * flux) and the fields are untouched.  Errors: MB_ERR_ARG (null context),
 * MB_ERR_CUDA. */
int mb_reset_probes(mb_ctx* ctx);

/* Advance n >= 0 steps like mb_step, but with direct launches bracketed by
 * CUDA events on the context's stream; synchronizes, then adds the summed
 * device time (ms) of each pass over the n steps to ms_out[0..3]: H pass,
 * fused E pass, point-probe DFT, face- and plane-probe DFTs (ms_out may be
 * NULL).  With the single-pass step (mb_set_single_pass) ms_out[0] is the
 * single-pass launches and ms_out[1] stays ~0. */
int mb_step_timed(mb_ctx* ctx, int n, double* ms_out);

/* Wait for the context's queued work (the probe launches on its second
 * stream included). */
int mb_synchronize(mb_ctx* ctx);

/* Steps taken so far. */
int mb_get_step(mb_ctx* ctx, int64_t* n);

/* Point-probe spectrum S(lam_k) = sum_c |E~_c(w_k)|^2 ((V s)^2/m^2) into
 * out_S (host, n_freq) and the wavelengths into out_lam (host, may be NULL). */
int mb_probe_spectrum(mb_ctx* ctx, int probe_id, double* out_S, double* out_lam);

/* Outward Poynting spectral density of face f (0..5 = x-, x+, y-, y+, z-, z+),
 * sum over its probe points of Re(E~_a H~_b^* - E~_b H~_a^*) dA (J s). */
int mb_face_spectrum(mb_ctx* ctx, int face, double* out_S, double* out_lam);

/* Electromagnetic energy U = 1/2 sum (eps0 eps_r |E|^2 + mu0 |H|^2) dx^3 (J)
 * of the stored fields, and, if out_flux6 != NULL, the energy (J) that has
 * left through each face of the interior box since creation: outward flux of
 * (E^n + E^{n+1})/2 on the face plane against H^{n+1/2} half a cell outside,
 * times dt, summed over steps (the exact discrete Poynting balance of the
 * box).  Returns MB_ERR_NONFINITE if any field value is NaN or Inf. */
int mb_energy(mb_ctx* ctx, double* out_U, double* out_flux6);

/* Only the six time-integrated face energies of mb_energy (J): summed on
 * the device, a 48-byte device-to-host read, no reduction over the grid.
 * Synchronizes. */
int mb_flux(mb_ctx* ctx, double* out_flux6);

/* The same six values, asynchronously: queued on the context's stream after
 * the work already queued; host_out6 (6 doubles, caller-owned) holds them
 * once the stream has passed this point (after mb_synchronize, or an event
 * recorded on the context's stream after this call).  In page-locked host
 * memory (cudaHostAlloc, cudaHostRegister, torch pin_memory) the summing
 * kernel writes them there directly; other memory gets a device-to-host
 * copy.  It does not wait for probes left running by mb_step (the face
 * energies are accumulated by the field step itself).  The buffer must stay
 * valid until then.
 * Device-side wait failures are reported by the next synchronizing call.
 * Errors: MB_ERR_ARG (null output), MB_ERR_CUDA. */
int mb_flux_async(mb_ctx* ctx, double* host_out6);

/* Diagnostic copy of the CPML memories of the slabs along one axis (0: x,
 * 1: y, 2: z) to host memory, SI units (FP64).  *count receives the number
 * of values (host_out may be NULL to query it; 0 without CPML).  Four planes
 * f of equal size: f = 0, 1 the E-update memories (A/m^2; x: Ey, Ez, y: Ex,
 * Ez, z: Ex, Ey), f = 2, 3 the H-update memories (V/m^2; x: Hy, Hz, y: Hx,
 * Hz, z: Hx, Hy), each the running convolution psi <- b psi + c dF/dw of the
 * derivative along the axis (Roden & Gedney 2000).  Index of slab layer s
 * (s = i for i < npml, i - n + 2 npml for i >= n - npml):
 *   x: ((f n_z + k) n_y + j) 2 npml + s,   y: ((f n_z + k) 2 npml + s) n_x + i,
 *   z: ((f zn + s) n_y + j) n_x + i with zn = 2 npml layers (s as above). */
int mb_get_cpml(mb_ctx* ctx, int axis, double* host_out, size_t* count);

/* Diagnostic copy of the context's gain-cell list (the cells whose material
 * byte has the gain bit, in increasing order, built on the device by
 * mb_set_material for the two-pass step's Lorentz blocks) to host memory.
 * *count receives the number of entries (host_out may be NULL to query it).
 * Errors: MB_ERR_STATE before mb_set_material. */
int mb_gain_list(mb_ctx* ctx, uint32_t* host_out, int64_t* count);

/* Diagnostic copy of the context's material bytes (n cells, x fastest; bits
 * 0..6: the id of the cell's eps_r value in order of first appearance in
 * the map, 0 for a dense map; bit 7: gain cell), as mb_set_material built
 * them on the device: equal to mb_material_map's.  Errors: MB_ERR_STATE
 * before mb_set_material. */
int mb_get_material(mb_ctx* ctx, uint8_t* host_out);

/* Copy one field (MB_EX..MB_N3) to / from host memory (n cells, SI units).
 * N0 is derived (N_a minus the other three) and cannot be set. */
int mb_get_field(mb_ctx* ctx, int which, float* host_out);
int mb_set_field(mb_ctx* ctx, int which, const float* host_in);

/* Copy one field, in the device's scaled units, into caller-owned device
 * memory dev_out (n floats); *scale (may be NULL) receives the factor that
 * turns it into SI.  N0 is not stored and is rejected. */
int mb_get_field_device(mb_ctx* ctx, int which, float* dev_out, double* scale);

/* Whole state (fields, CPML memory, probe accumulators, step count) as an
 * opaque host blob.  Call with host_blob == NULL to query *bytes. */
int mb_save_state(mb_ctx* ctx, void* host_blob, size_t* bytes);
int mb_load_state(mb_ctx* ctx, const void* host_blob, size_t bytes);

/* Time the candidate thread-block shapes of the two field passes on this
 * grid (the state is saved and restored around the trials) and keep the
 * fastest.  The choice is cached per grid shape for the process. */
int mb_autotune(mb_ctx* ctx);

/* Launch shape of the H pass and of the E pass, as {variant, bx, by, bz}:
 * variant 0 = one thread per cell in (bx, by, bz) blocks; 1 = 2-D (bx, by)
 * blocks whose threads each walk bz planes along z; 2 (n_x a multiple of
 * 16) = the same walk with the planes staged in shared memory by bulk
 * tensor copies (TMA), tiles 32x4, 32x8, 64x4, 64x8, 128x2, 128x4;
 * 3 (n_x a multiple of 4) = the walk over quads of 4 x-cells with 16-byte
 * accesses, bx counting quads.  Every variant gives the same bits.  Read
 * the current choice or set one (bx a multiple of 32, at most 512 threads,
 * 256 for variant 3). */
int mb_get_tuning(mb_ctx* ctx, int tune_h[4], int tune_e[4]);
int mb_set_tuning(mb_ctx* ctx, const int tune_h[4], const int tune_e[4]);

/* Single-pass step: the H half-step, the gain cells' Lorentz / Langevin
 * update and the E / population update of one time step (the step of the
 * "Simulations" paragraph) in one launch.  It reads the current copy of E,
 * H and the CPML memories and writes a second copy of them (allocated on
 * the first such step: 24 bytes per cell plus the CPML memories), which
 * becomes the current one; every call of this header (fields, snapshots,
 * probes, energy, the adjoint) follows the current copy, so the alternation
 * is invisible to the caller.  P, J and the populations are updated in
 * place.  Fields, probes and energy equal
 * the two-pass step's bit for bit (the face-flux sums agree to the FP32
 * rounding of their partial sums).  tune = {on (0 or 1), bx, by, kz}: tiles of bx x by columns
 * (32x4, 32x8, 64x4 or 64x8) walking kz planes; needs n_x a multiple of 16.
 * mb_autotune selects it when it is the faster.  Errors: MB_ERR_ARG (bad
 * tile or grid), MB_ERR_OOM (second copy). */
int mb_get_single_pass(mb_ctx* ctx, int tune[4]);
int mb_set_single_pass(mb_ctx* ctx, const int tune[4]);

/* Kernel launches queued per step by mb_step, and in total so far. */
int mb_launch_stats(mb_ctx* ctx, int* per_step, int64_t* total);

/* Test hook: the n-th device allocation made by mb_create or by the
 * single-pass step's second copy from now on (n = 0: the next one) fails as
 * if the device were out of memory (MB_ERR_OOM, nothing leaked); n < 0
 * switches the injection off.  Process-wide. */
void mb_debug_fail_alloc(int n);

/* Device bytes the context holds. */
int mb_device_bytes(mb_ctx* ctx, size_t* bytes);

/* Diagnostic (host only, no device work): the coefficient tables a context
 * with these arguments steps with (p NULL: defaults), in device units.
 * out_cpml (4 (n_x + n_y + n_z) floats): per axis x, y, z the CPML b and c of
 * the E update (at cell positions i) and of the H update (at i + 1/2), each
 * n_w values, zero outside the layers.  out_gain (20 floats, zero when
 * N_a = 0): cJ1, cJE, cJP, cJN, nfloor, g[3], G[3][3] (row-major), mk[3] of
 * the gain update n' = n + g + G n + mk S, n = (N1, N2, N3)/N_a.  out_E0: the
 * field scale E0 (V/m).  Errors: MB_ERR_ARG. */
int mb_host_tables(const int grid[3], double dx, double dt, const mb_params* p, double N_a,
                   double pump, float* out_cpml, float* out_gain, double* out_E0);

/* Diagnostic (host only, no device work): the material map mb_set_material
 * builds from eps_map and gain_mask (host, n cells each), with at most
 * max_threads host threads.  out_mat (n bytes): bits 0..6 the id of the
 * cell's eps_r value (ids in order of first appearance), bit 7 set for a gain
 * cell when gain_on; out_glist (capacity n): the gain cells' indices in
 * increasing order, out_n_gain of them; out_lut_eps (capacity 128): the
 * distinct values in id order, out_n_values of them; *out_dense = 1 when there
 * are more than 128 values (every id 0, no values listed).  Errors:
 * MB_ERR_ARG (null pointer, n < 1), MB_ERR_MATERIALS (a value not finite or
 * below 1), MB_ERR_OOM. */
int mb_material_map(const float* eps_map, const uint8_t* gain_mask, int64_t n, int gain_on,
                    int max_threads, uint8_t* out_mat, uint32_t* out_glist, int64_t* out_n_gain,
                    float* out_lut_eps, int* out_n_values, int* out_dense);

/* Diagnostic: evaluate the device's Philox4x32-10 (the generator of the
 * Langevin force, Salmon et al. SC'11) on n counters.  ctr (host, 4n words),
 * key (host, 2 words), out (host, 4n words).  Runs one kernel on the current
 * device and synchronizes.  Errors: MB_ERR_ARG, MB_ERR_CUDA. */
int mb_philox4x32_10(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, int n);

/* ------------------------------------------------------------------------
 * Batched ensemble.  The paper's pump sweep ("spectra for two pumping
 * levels", Fig. 2b,c; linewidth versus pump, Fig. 5b) and disorder
 * averages need many realizations; a batch advances B of them, on grids of
 * any (uneven) sizes, together, in one of two modes.  MB_BATCH_PERSISTENT:
 * every mb_batch_step launch runs n steps of all instances in one
 * persistent cooperative kernel (per step: all H tiles and gain cells, a
 * grid barrier, all E tiles, a grid barrier), replayed from a CUDA graph.
 * MB_BATCH_CONCURRENT: each instance takes its own steps (its tuned
 * single-context launches and graphs, as mb_step) on one of several
 * streams that run side by side, forked from and joined back into the
 * batch's stream; small instances then fill the GPU together.
 * mb_batch_autotune times both and keeps the faster; the results are the
 * same bits either way.  Each instance is an ordinary context (obtained with
 * mb_batch_instance) whose fields, probes and read-outs behave as with
 * mb_step — the fields are bit-identical to stepping the instance alone.
 * Supported inside a batch: point probes, sources, the face flux and energy;
 * mb_batch_step returns MB_ERR_STATE when a member has face or plane probes, has no
 * material yet, or was stepped outside the batch.  A barrier that waits
 * longer than ~1 s makes the launch end and mb_batch_synchronize return
 * MB_ERR_TIMEOUT. */
typedef struct mb_batch mb_batch;

/* B instances; grids holds 3 ints per instance.  Errors as mb_create. */
int mb_batch_create(mb_batch** out, int B, const int* grids, double dx, double dt,
                    const mb_params* p, void* cuda_stream);
int mb_batch_destroy(mb_batch* batch);

/* Material, pump and noise seed of instance b (see mb_set_material). */
int mb_batch_set_instance(mb_batch* batch, int b, const float* eps_map,
                          const uint8_t* gain_mask, double N_a, double pump, uint64_t seed);

/* The context of instance b (owned by the batch; do not destroy it).  Probes
 * and sources added to it, and its read-outs, work as for a single context;
 * step it only through the batch. */
int mb_batch_instance(mb_batch* batch, int b, mb_ctx** ctx);

/* Advance every instance n steps (asynchronous). */
int mb_batch_step(mb_batch* batch, int n);

/* Wait for the batch's work; MB_ERR_TIMEOUT if a grid barrier gave up. */
int mb_batch_synchronize(mb_batch* batch);

/* Time the candidate tile shapes of the persistent kernel, tune each
 * instance's own launches (mb_autotune), time the two modes over a few
 * steps (states are saved and restored around every trial) and keep the
 * fastest shape and mode. */
int mb_batch_autotune(mb_batch* batch);

#define MB_BATCH_PERSISTENT 0
#define MB_BATCH_CONCURRENT 1

/* Mode of mb_batch_step (MB_BATCH_PERSISTENT after creation).  Errors:
 * MB_ERR_ARG (null batch or output, unknown mode). */
int mb_batch_set_mode(mb_batch* batch, int mode);
int mb_batch_get_mode(mb_batch* batch, int* mode);

/* Tile shape of the persistent kernel: out3 = {bx, by, kz} (a block of bx x by
 * threads walks kz z-planes of one tile). */
int mb_batch_get_tuning(mb_batch* batch, int* out3);

/* ------------------------------------------------------------------------
 * One grid split along z into slabs.  The paper runs its FDTD grid
 * "distributed on (typically) 256 processors" ("Simulations" paragraph);
 * here each slab is a context of its own (on one GPU or on several) and
 * neighbouring slabs exchange one plane each way per step.
 *
 * A slab context holds the planes z_begin .. z_end-1 of a grid of grid[2]
 * planes (its own planes) plus a ghost plane next to each neighbour: local
 * plane 0 is plane z_begin - 1 when z_begin > 0, and the last local plane
 * is plane z_end when z_end < grid[2].  All other calls address the
 * context's local planes (host arrays of mb_set_material, mb_get_field,
 * probe and source cells are n_x x n_y x local n_z, ghost planes included;
 * mb_set_material must be given the whole grid's values on the ghost planes
 * too).  The whole grid's boundaries hold: PEC walls and the CPML profile of
 * the whole grid along z, the Langevin noise keyed by each cell's index in
 * the whole grid (so a split run draws the same noise as the whole grid),
 * the face-flux box of the whole grid cut to the own planes, mb_energy over
 * the own planes only, face probes (mb_add_face_probes) on the whole grid's
 * lattice of points cut to the own planes (a z face is kept by the slab
 * owning the plane below it), so that a face spectrum of the whole grid is
 * the sum of the slabs' mb_face_spectrum.  The adjoint is not available on
 * a slab (MB_ERR_STATE).
 *
 * Step protocol (what makes the split run equal, cell by cell, to the whole
 * grid): before every step, for each pair of neighbouring slabs A (below)
 * and B (above), mb_halo_pack(A, 1, buf) then mb_halo_unpack(B, 0, buf), and
 * mb_halo_pack(B, 0, buf') then mb_halo_unpack(A, 1, buf'); then mb_step(ctx,
 * 1) on every slab.  A packed plane is the whole time-n state of a boundary
 * plane (E, H, P, J, populations, x / y CPML memories).  The own cells'
 * fields then equal the whole grid's bit for bit; the FP64 read-outs (energy,
 * face flux) summed over the slabs equal the whole grid's up to the order of
 * summation.  mb_step(ctx, n > 1) without exchanges in between leaves the
 * boundary planes wrong.
 * ------------------------------------------------------------------------ */

/* Create the slab context of planes [z_begin, z_end) of a grid[0] x grid[1]
 * x grid[2] grid; other arguments as mb_create.  A cut plane z_begin > 0 or
 * z_end < grid[2] must lie in [npml + 1, grid[2] - npml - 1] (ghost planes
 * outside the z-CPML), and the whole grid must have fewer than 2^32 cells
 * (the noise counter).  Errors: as mb_create, MB_ERR_ARG for a bad range or
 * cut. */
int mb_create_slab(mb_ctx** out, const int grid[3], int z_begin, int z_end, double dx,
                   double dt, const mb_params* p, void* cuda_stream);

/* info = (whole grid's n_z, whole-grid plane of local plane 0, first own
 * local plane, one past the last own local plane); for a context made by
 * mb_create: (n_z, 0, 0, n_z). */
int mb_slab_info(mb_ctx* ctx, int info[4]);

/* Bytes of one packed boundary plane: 4 (15 n_x n_y + 8 npml (n_x + n_y)). */
int mb_halo_bytes(mb_ctx* ctx, size_t* bytes);

/* Pack the state of the lowest (side 0) or highest (side 1) own plane into
 * d_buf, a device buffer of mb_halo_bytes on the context's device; queued
 * on the context's stream.  Errors: MB_ERR_ARG, MB_ERR_STATE (not a slab). */
int mb_halo_pack(mb_ctx* ctx, int side, void* d_buf);

/* Write a neighbour's packed plane (d_buf, as mb_halo_pack wrote it) into
 * the ghost plane below (side 0) or above (side 1); queued on the context's
 * stream, which must be ordered after the pack.  Errors: MB_ERR_ARG,
 * MB_ERR_STATE (not a slab, or no ghost plane on that side). */
int mb_halo_unpack(mb_ctx* ctx, int side, const void* d_buf);

/* ------------------------------------------------------------------------
 * Adjoint gradient of emitted energy.  The paper observes emission through
 * probe planes ("Simulations" paragraph, spectra of Figs. 1-2) and varies the
 * pump (Figs. 2, 5); this call differentiates that read-out.  Objective: the
 * energy (J) crossing the plane z = z_plane dx in +z during the next n_steps
 * steps, over the interior rectangle (the CPML-free x, y range), with the
 * same discrete Poynting pairing as the face flux ((E^n + E^{n+1})/2 on the
 * plane against H^{n+1/2} half a cell below it); z_plane < 0 selects the
 * box's +z face, n_z - npml.
 *
 * The context advances n_steps exactly as mb_step would (probes and flux
 * included); then a reverse-time discrete adjoint of the FP32 step runs back
 * over the window.  Forward checkpoints are kept every ckpt_every steps
 * (<= 0: 200); each segment is recomputed and its states stored (48 bytes
 * per cell per step) before its reverse sweep.  Noise and sources are held
 * fixed: the gradient is that of the realization with this seed.
 *   d_grad_eps  device array of n_cells floats (x fastest) or NULL:
 *               dJ/d eps_r of every cell, in J per unit eps_r (each cell's
 *               eps_r taken as its own variable), accumulated in FP64;
 *   grad_pump   host double or NULL: dJ/dW_p in J s;
 *   J_out       host double or NULL: the objective J.
 * Device memory for checkpoints, the segment store and the adjoint fields is
 * allocated for the call and freed before it returns.  Synchronous.
 * Errors: MB_ERR_ARG (n_steps < 1, plane outside 1 <= p < n_z), MB_ERR_STATE
 * (no material), MB_ERR_OOM, MB_ERR_CUDA. */
int mb_adjoint_energy_zface(mb_ctx* ctx, int n_steps, int ckpt_every, int z_plane,
                            float* d_grad_eps, double* grad_pump, double* J_out);

/* Self-test of the bounded device waits (no counterpart in the paper): runs
 * the batched kernel's grid barrier against a block that never arrives
 * (which = 0, a cooperative grid of up to 8 blocks) or the TMA kernels'
 * mbarrier wait against a transaction that never completes (which = 1, one
 * block), with at most `limit` polls (1 .. 2^22), and stores in *gave_up the
 * number of blocks whose wait ended unfulfilled (the grid's size, or 1).
 * Nothing faults or hangs: the waits end by themselves and the device stays
 * usable.  Synchronizes the device.  Errors: MB_ERR_ARG, MB_ERR_CUDA. */
int mb_selftest_bounded_waits(int which, int limit, int* gave_up);

/* ------------------------------------------------------------------------
 * Theory side: the bound state phi(tau) > 0 of
 *     -phi'' + tau^2 phi + phi^3 = E phi        (the paper's Eq. g5)
 * for each eigenvalue E[q] > 1 (bound states exist above threshold), on
 * n_grid points tau_i = -L + i h, i = 1..n_grid, h = 2L/(n_grid + 1),
 * L = sqrt(E) + 8, phi(+-L) = 0, second-order differences, solved in FP64 on
 * the GPU by Newton's method (one thread per eigenvalue).  Outputs (host
 * arrays of nE doubles): w_phi[q], the standard deviation of |phi~|^2 in the
 * frequency Omega / 2 pi, and p_phi[q] = |phi~(0)|^2 / (4 pi^2), with phi~
 * the Fourier transform of phi — the normalised spectral waist and peak of
 * the paper's Figs. 3 and 5 (W = w_phi sqrt(kappa) / (p^{1/4} t_g), S_p =
 * t_g^2 p_phi / gamma_S).  phi_out (host, nE x n_grid doubles) may be NULL.
 * Synchronous.  Errors: MB_ERR_ARG (E <= 1 or not finite, n_grid outside
 * 16..2^20), MB_ERR_STATE (Newton did not reach a bound state), MB_ERR_OOM,
 * MB_ERR_CUDA. */
int mb_gp_features(const double* E, int nE, int n_grid, double* w_phi, double* p_phi,
                   double* phi_out);

/* The paper has no counterpart of this call: it is a service for callers
 * that cannot allocate device memory — code running while a framework's
 * caching allocator owns the device memory, code that must not pay the
 * device-wide synchronisation of cudaMalloc / cudaFree, code under a
 * per-process memory limit.  It computes what mb_energy reduces, from
 * caller-owned device arrays, without allocating anything:
 *   d_out[0] = sum_c (w_c (Ex^2 + Ey^2 + Ez^2) + Hx^2 + Hy^2 + Hz^2)   (FP64)
 *   d_out[1] = 1.0 if any value was NaN/Inf, else 0.0
 * with w_c = d_eps_r[c] (d_eps_r may be NULL: w = 1).  With the context's
 * scaled fields (mb_get_field_device) and eps_r, U = eps0 E0^2 dx^3 d_out[0]/2
 * where E0 is the scale of MB_EX.  All pointers are device pointers the
 * caller owns (n cells of float; d_out 2 doubles); the work is queued on
 * cuda_stream (NULL: the legacy default stream) and not waited for.
 * Scratch: a static device array of 8192 partial sums (64 KB) that every GPU
 * loading the library holds until exit; hence ncell <= 67,108,864
 * (MB_ERR_ARG beyond).  The first call on a device, with that device
 * current, looks up the array's device address; make that first call before
 * any stream capture.  The address belongs to the device's context: after a
 * device reset the next call looks it up again (also before any capture).  Calls share the array: calls that overlap on the GPU
 * (different streams or threads) race and must be serialised by the caller.
 * Errors: MB_ERR_ARG, MB_ERR_CUDA; the message is mb_last_error(NULL). */
int mb_energy_sum_noalloc(const float* d_ex, const float* d_ey, const float* d_ez,
                          const float* d_hx, const float* d_hy, const float* d_hz,
                          const float* d_eps_r, int64_t ncell, double* d_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MB_FDTD_H */
