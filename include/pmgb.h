/*
 * pmgb - particle-mesh N-body force evaluation and BullFrog time integration
 * on one GPU (GB300, sm_103a).  C ABI of libpmgb.so.
 *
 * Method: "DISCO-DJ II: a differentiable particle-mesh code for cosmology"
 * (arXiv:2510.05206).  Each entry point cites the section of the paper that
 * defines the operation.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Units: box size L in Mpc/h, wavenumbers in h/Mpc, displacements in Mpc/h,
 *   velocities are growth-factor-time velocities V = dX/dD (Sec. 2.4) in Mpc/h.
 * - D is normalised as D ~ a for a -> 0 (Sec. 2.4, footnote on BullFrog).
 * - A handle serves `batch` independent simulations ("slots") of identical
 *   size.  Particle arrays are float32, device memory, caller-owned, laid out
 *   [slot][component x,y,z][particle], particle i = (iz*np + iy)*np + ix on the
 *   Lagrangian lattice q = (ix, iy, iz) L / np.  disp = X - q (Sec. 2.2).
 * - Meshes are float32 [slot][z][y][x]; node j sits at r_j = j L / n.
 * - Every call that launches work is asynchronous on the handle's stream
 *   (pm_init / pm_set_stream) unless its comment says it synchronises.  No call
 *   allocates device memory after pm_init, except where stated.
 * - Return value: PM_OK (0) or a negative PM_ERR_* code; pm_last_error() then
 *   holds a one-line message.  No C++ exception crosses the ABI.
 * - A handle is not thread-safe; distinct handles may be used concurrently.
 * - Sizes: n_part, n_mesh and P(k) meshes are powers of two in [16, 1024].
 */
#ifndef PMGB_H
#define PMGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PM_OK 0
#define PM_ERR_ARG (-1)         /* invalid argument or configuration */
#define PM_ERR_CUDA (-2)        /* a CUDA runtime call or kernel launch failed */
#define PM_ERR_OOM (-3)         /* device allocation failed */
#define PM_ERR_STATE (-4)       /* call not valid in the handle's current state */
#define PM_ERR_UNSUPPORTED (-5) /* option combination not implemented */

typedef struct pm_handle pm_handle;

/* Run configuration (Table 4 of the paper lists the defaults it uses). */
typedef struct pm_config {
    int32_t n_part;      /* particles per dimension, N = n_part^3 */
    int32_t n_mesh;      /* PM mesh cells per dimension (Table 4 res_pm) */
    double box;          /* L [Mpc/h] */
    int32_t order;       /* mass-assignment kernel (Table 1): 2 = CIC, 3 = TSC, 4 = PCS */
    int32_t interlace;   /* 0, or 1 = one extra grid shifted by half a cell (Sec. 2.8) */
    int32_t grad_order;  /* gradient kernel (Table 2): 0 = i k, 2/4/6 = finite difference; default 4 */
    int32_t lap_order;   /* Laplacian kernel (Table 2): 0 = -k^2, 2/4/6; default 0 */
    double omega_m;      /* flat LambdaCDM, Omega_L = 1 - Omega_m */
    double h;            /* H0 / (100 km/s/Mpc), enters the BBKS shape Gamma = Omega_m h */
    double n_s;          /* primordial spectral index */
    double sigma8;       /* normalisation of the linear spectrum at a = 1 */
    double a_ini;        /* initial scale factor */
    double a_end;        /* final scale factor */
    int32_t n_steps;     /* number of DKD steps */
    int32_t stepper;     /* 0 = BullFrog (default), 1 = FastPM (Sec. 2.4) */
    int32_t time_var;    /* 0 = steps uniform in D (default), 1 = uniform in a (Sec. 2.4) */
    int32_t zero_corner; /* 1 = zero initial modes with |k| > k_Nyquist (App. A.3; default 1) */
    int32_t batch;       /* number of simulation slots served by the handle (>= 1) */
    int32_t pk_mesh_max; /* largest mesh pm_power_spectrum may use (0 = n_mesh) */
    int32_t deconvolve;  /* 1 = divide the force's density spectrum by the squared mass
                            assignment kernel, prod_c W^(k_c)^2 with W^ = sinc^p(k/2) of
                            Table 1 (Sec. 2.5, deconvolution of the interpolation kernel;
                            Table 4 `deconvolve`, default 0) */
    int32_t lpt_order;   /* initial conditions: 1 = Zel'dovich (default, also 0), 2 = 2LPT
                            (Sec. 2.2, Eq. LPT at n = 2 with D^n growth: Psi = D psi1 + D^2 psi2,
                            V = psi1 + 2 D psi2; Table 4 `nlpt_order_ics`) */
    int32_t nufft;       /* 1 = force by the NUFFT (Sec. 2.5): exponential-of-semicircle kernel of
                            width 5 (5^3 taps) on a grid of 2 n_mesh cells per dimension, modes
                            |m| < n_mesh/2 per axis, deconvolved by the kernel's transform twice;
                            `order` is then unused and grad_order = lap_order = 0 (exact kernels),
                            interlace = deconvolve = 0 are required; forward only (no adjoint,
                            JVP or stage calls); default 0 */
} pm_config;

/* Fills *cfg with the defaults: CIC, no interlacing, 4th-order gradient, exact
 * Laplacian, Omega_m 0.3, h 0.7, n_s 0.96, sigma8 0.8, a 0.02 -> 1, 6 BullFrog
 * steps uniform in D, corner modes zeroed, no deconvolution, Zel'dovich ICs, batch 1;
 * n_part = n_mesh = 64, L = 256. */
void pm_config_default(pm_config* cfg);

/* Device bytes pm_init will allocate for cfg (for admission control). */
int pm_workspace_bytes(const pm_config* cfg, size_t* bytes);

/* Validates cfg, computes the FP64 growth and step tables on the host (App. B,
 * Sec. 2.4), allocates the workspace (meshes, spectra, tables) with cudaMalloc
 * and uploads the tables.  stream: a cudaStream_t (NULL = legacy default
 * stream).  Synchronises the device.  On failure *out is NULL and
 * pm_last_error(NULL) explains why. */
int pm_init(const pm_config* cfg, void* stream, pm_handle** out);

/* Frees the handle and its workspace (synchronises its stream). NULL is a no-op. */
void pm_destroy(pm_handle* h);

/* Message of the last failing call on h (h = NULL: the last failing pm_init). */
const char* pm_last_error(const pm_handle* h);

/* Switches the stream subsequent calls enqueue on. */
int pm_set_stream(pm_handle* h, void* stream);

/* Copies the handle's per-step coefficient table to host memory `out`
 * (n_steps rows of 7 doubles: tau1, tau2, alpha, beta, D_half, D_n, D_{n+1};
 * Eq. dkd and the BullFrog/FastPM alpha, beta of Sec. 2.4).  cap = rows available. */
int pm_step_table(const pm_handle* h, double* out, int32_t cap);

/* Same table computed from a configuration alone, on the host (no GPU work,
 * no allocation): out receives cfg->n_steps rows of 7 doubles. */
int pm_host_step_table(const pm_config* cfg, double* out, int32_t cap);

/* Growth factors of the handle's cosmology at scale factor a (host, FP64):
 * out[0] = D(a), out[1] = E(a), out[2] = dE/dD (App. B). */
int pm_growth(const pm_handle* h, double a, double* out);

/* Zel'dovich initial conditions (Sec. 2.2, Sec. 2.4) for every slot:
 * noise: unit-variance white noise [slot][n_part^3] (device, real space, same
 * lattice order as the particles).  delta_lin(a=1)^ = noise^ sqrt(P(k) N / L^3),
 * P = BBKS spectrum normalised to sigma8; psi1^ = i k / k^2 delta_lin^ / D(1)
 * with k = 0, every Nyquist plane and (zero_corner) |k| > k_Ny set to zero;
 * vel = psi1, disp = D(a_ini) psi1.
 * With cfg.lpt_order = 2 (2LPT, Sec. 2.2 Eqs. LPT / helmholtz / LPT_L_and_T at
 * n = 2): psi2 = Lap^-1 grad L2, L2 = -(3/7) (1/2)(psi1_i,i psi1_j,j - psi1_i,j psi1_j,i),
 * formed on the lattice grid with exact i k / -k^2 kernels, zero at k = 0 and on
 * every Nyquist plane; disp = D psi1 + D^2 psi2, vel = psi1 + 2 D psi2 (D = D(a_ini)).
 * 2LPT uses the force-mesh workspace as scratch (sized for it by pm_init). */
int pm_ic_zeldovich(pm_handle* h, const float* noise, float* disp, float* vel);

/* Same for one slot: noise, disp and vel point at that slot's data. */
int pm_ic_zeldovich_slot(pm_handle* h, int32_t slot, const float* noise, float* disp, float* vel);

/* One DKD step (Eq. dkd) of index `step` (0-based) for every slot:
 * X_half = X + tau1 V; V <- alpha V + beta A(X_half); X <- X_half + tau2 V, with
 * A = -grad Lap^-1 delta / D_half^2 from the PM force (Sec. 2.5: deposit,
 * real FFT, Green's function and gradient kernels, inverse FFTs, interpolation
 * with the same kernel).  disp, vel are updated in place. */
int pm_step(pm_handle* h, float* disp, float* vel, int32_t step);

/* Steps step_begin .. step_end-1 (0 <= begin <= end <= n_steps). */
int pm_run(pm_handle* h, float* disp, float* vel, int32_t step_begin, int32_t step_end);

/* Continuous batching: sets, on the host, which step each slot takes next.
 * n_steps[slot] = total steps of the simulation in that slot (its own
 * coefficient table over [a_ini, a_end]), step[slot] = index of its next step,
 * or < 0 for an idle slot.  The coefficients are copied to the device on the
 * handle's stream; pm_step_slots reads them there. */
int pm_set_slots(pm_handle* h, const int32_t* n_steps, const int32_t* step);

/* One step for every active slot, each with the coefficients set by
 * pm_set_slots.  Launches kernels and memsets only (CUDA-graph capturable). */
int pm_step_slots(pm_handle* h, float* disp, float* vel);

/* Binned power spectrum of the particles at X = q + disp for every slot
 * (Sec. 2.9 analysis; CIC density on an n_mesh^3 mesh, delta = rho M/N - 1):
 * P(k_b) = (L^3/M^2) <|delta^_k|^2> over the modes with (b+1/2) k_F <= |k| < (b+3/2) k_F,
 * k_F = 2 pi / L; no deconvolution, no shot-noise subtraction.  Accumulated in
 * FP64.  Outputs are HOST arrays [slot][n_bins]: k (mean |k| of the bin), pk,
 * n_modes (modes of the full n^3 grid).  Synchronises the stream. */
int pm_power_spectrum(pm_handle* h, const float* disp, int32_t n_mesh, int32_t n_bins, double* k, double* pk,
                      int64_t* n_modes);

/* pm_power_spectrum in two halves, for callers that keep the GPU busy while
 * results travel.  pm_power_spectrum_async enqueues the deposit, transform and
 * binning on the handle's stream and returns without synchronising: bin_sums is
 * a DEVICE array [slot][n_bins] (caller-owned) that receives, per bin, the FP64
 * sum over its modes of w |rho^_k|^2 (w = 2 for the half-spectrum modes that
 * stand for +-k).  The work is stream-ordered: bin_sums is complete once the
 * stream has passed it (an event recorded after the call, or any later
 * synchronisation).
 * pm_power_spectrum_finish turns a HOST copy of those sums into the outputs of
 * pm_power_spectrum (k, pk, n_modes, host arrays [slot][n_bins]); it launches
 * nothing and does not touch the device. */
int pm_power_spectrum_async(pm_handle* h, const float* disp, int32_t n_mesh, int32_t n_bins, double* bin_sums);
int pm_power_spectrum_finish(pm_handle* h, int32_t n_mesh, int32_t n_bins, const double* bin_sums, double* k,
                             double* pk, int64_t* n_modes);

/* Forward mode of pm_power_spectrum: with the tangent tdisp of disp, dpk[slot][bin]
 * = (L^3/M^2) <2 Re(conj(delta^) delta'^)> over the bin's modes (delta' the CIC
 * density tangent of X = q + disp along tdisp, times M/N); k, pk, n_modes as
 * pm_power_spectrum (which it also runs).  Synchronises the stream. */
int pm_power_spectrum_jvp(pm_handle* h, const float* disp, const float* tdisp, int32_t n_mesh, int32_t n_bins,
                          double* k, double* pk, double* dpk, int64_t* n_modes);

/* Density contrast delta = rho M / N - 1 of X = q + disp on an n_mesh^3 mesh with
 * kernel `order` (Table 1), every slot: delta [slot][n_mesh^3] device. */
int pm_density(pm_handle* h, const float* disp, int32_t n_mesh, int32_t order, float* delta);

/* Force field g = -grad Lap^-1 delta on the handle's mesh (Sec. 2.5, Table 2
 * kernels; k = 0 and each component's own Nyquist plane zeroed):
 * delta [slot][n_mesh^3] -> force [slot][3][n_mesh^3] (device). */
int pm_force_mesh(pm_handle* h, const float* delta, float* force);

/* Interpolation with the handle's kernel (Sec. 2.5): acc[slot][c][i] =
 * sum_j force[slot][c][j] W(r_j - X_i), X = q + disp. */
int pm_interp(pm_handle* h, const float* disp, const float* force, float* acc);

/* Adjoint method (Sec. 2.7, Table 5) with the scatter/gather pullbacks of
 * App. C, for every slot, in place and with memory independent of the number
 * of steps: on entry (disp, vel) is the state after step_end steps and
 * (adj_disp, adj_vel) = (dL/dPsi, dL/dV) there; steps step_end-1 .. 0 run
 * backwards (primal drift back, adjoint drift, force recomputation, primal
 * kick back, adjoint kick through the VJP of A, velocity cotangent rescale,
 * drift back, adjoint drift).  On return (disp, vel) is the reintegrated
 * initial state and (adj_disp, adj_vel) the cotangents of the initial state.
 * Single grid only (interlace = 0, else PM_ERR_UNSUPPORTED).  Allocates three
 * adjoint meshes per slot on its first call. */
int pm_adjoint(pm_handle* h, float* disp, float* vel, float* adj_disp, float* adj_vel, int32_t step_end);

/* Forward mode (Jacobian-vector products; the tangent counterpart of App. C's
 * scatter/gather derivatives): advances the state (disp, vel) and a tangent
 * (tdisp, tvel), same layout, through steps [step_begin, step_end) of the DKD
 * stepper.  Per step: X_half and X'_half = X' + tau1 V'; the density of X_half
 * and its tangent rho'_j = sum_i X'_half,i . grad_X W(r_j - X_i); the force
 * operator applied to both (it is linear); A = gather(g) and
 * A' = gather(g') + X'_half . grad gather(g); V' <- alpha V' + kick A', X' <- X'_half
 * + tau2 V'.  Tangent ICs come from pm_ic_zeldovich on the tangent noise (the ICs
 * are linear in the noise).  Single grid only (interlace = 0, else
 * PM_ERR_UNSUPPORTED).  Allocates a tangent density and force mesh per slot on
 * its first call. */
int pm_jvp(pm_handle* h, float* disp, float* vel, float* tdisp, float* tvel, int32_t step_begin, int32_t step_end);

/* Pullback through the Zel'dovich initial conditions: with psi1* = D(a_ini)
 * adj_disp + adj_vel, adj_noise = sum_c F_c^T psi1*_c (F_c: noise -> psi1_c);
 * dsigma8 (host [slot], may be NULL) = <adj_noise, noise> / sigma8, since psi1
 * is proportional to sigma8.  Synchronises the stream when dsigma8 != NULL.
 * Zel'dovich ICs only (lpt_order = 2: PM_ERR_UNSUPPORTED). */
int pm_ic_adjoint(pm_handle* h, const float* noise, const float* adj_disp, const float* adj_vel, float* adj_noise,
                  double* dsigma8);

/* Pullback of pm_density w.r.t. positions (App. C, scatter VJP w.r.t.
 * positions): adj_disp = (M/N) sum_j dL_ddelta_j d/dX W(r_j - X) (overwritten). */
int pm_density_vjp(pm_handle* h, const float* disp, int32_t n_mesh, int32_t order, const float* dL_ddelta,
                   float* adj_disp);

/* Phase timing.  enable != 0 starts recording a CUDA event pair around every
 * phase the handle enqueues (and resets the counters); 0 stops.  Phases:
 * 0 deposit, 1 forward x FFT, 2 forward y FFT, 3 z FFT with the Fourier-space
 * operator, 4 inverse y FFT, 5 inverse x FFT, 6 interpolation + kick + drift,
 * 7 Zel'dovich ICs, 8 P(k), 9 adjoint spectral passes, 10 interpolation + kick + drift
 * fused with the next step's deposit (reserved), 11 real-space gradient stencil.
 * Kernel launches are counted always. */
int pm_profile(pm_handle* h, int32_t enable);

/* Synchronises the stream and returns, per phase (cap >= 12 entries), the summed
 * event time in ms, the number of timed phase instances and the kernel launches. */
int pm_profile_read(pm_handle* h, double* ms, int64_t* calls, int64_t* launches, int32_t cap);

/* End-to-end run from HOST buffers: copies noise [slot][N] from host memory,
 * computes the Zel'dovich ICs and all n_steps steps, and copies disp and vel
 * [slot][3][N] back to host memory.  Allocates device state buffers on its
 * first call (owned by the handle).  Synchronises the stream. */
int pm_simulate_host(pm_handle* h, const float* noise, float* disp, float* vel);

/* The whole analysis step from HOST buffers: copies noise [slot][N] from host
 * memory, computes the Zel'dovich (or 2LPT) ICs, all n_steps steps and the
 * binned power spectrum of the final positions (as pm_power_spectrum: n_mesh,
 * n_bins, HOST outputs k, pk, n_modes [slot][n_bins]).  The particle state stays
 * on the device in the handle's buffers (shared with pm_simulate_host; allocated
 * on the first call of either).  Synchronises the stream. */
int pm_simulate_pk_host(pm_handle* h, const float* noise, int32_t n_mesh, int32_t n_bins, double* k, double* pk,
                        int64_t* n_modes);

/* Largest mesh pm_power_spectrum_static accepts (cells per dimension). */
#define PM_STATIC_PK_MAX_MESH 64

/* Power spectrum for callers that cannot allocate device memory (host
 * callbacks or pipelines that forbid cudaMalloc, plugins whose host owns every
 * allocation, processes whose device budget is already committed).  The paper
 * has no counterpart: it is the estimator of pm_power_spectrum (same bins and
 * normalisation, CIC, one simulation) without a handle.
 * disp: device [3][n_part^3] displacements (the particle layout above),
 * n_part a power of two in [16, 1024], box > 0, n_mesh a power of two in
 * [16, PM_STATIC_PK_MAX_MESH], n_bins in [1, n_mesh/2]; stream: cudaStream_t
 * (NULL = legacy default stream); k, pk, n_modes: HOST arrays of n_bins.
 * Allocates nothing: its ~2.4 MB of scratch is one file-scope __device__ array
 * that every GPU which loads libpmgb holds until the process exits.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * Every call reuses the same array and clears what must start at zero, so calls
 * that overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Synchronises the stream.  Returns PM_ERR_ARG for
 * sizes outside the limits (use the handle API for larger meshes) and
 * PM_ERR_CUDA if a CUDA call fails. */
int pm_power_spectrum_static(const float* disp, int32_t n_part, double box, int32_t n_mesh, int32_t n_bins,
                             void* stream, double* k, double* pk, int64_t* n_modes);

#ifdef __cplusplus
}
#endif

#endif /* PMGB_H */
