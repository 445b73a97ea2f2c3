// Host-side launchers of the PM kernels (internal to libpmgb; the public C ABI
// is include/pmgb.h).  Every launcher enqueues on the given stream and returns
// 0, or -1 for an unsupported size.
#pragma once
#include <cuda_runtime.h>
#include "pm_common.cuh"

struct PmZPass {
    const float2* in[3];
    float2* out[6];
    long long slot_stride;
    const float2* tw;
    const float* lap1;
    const float* grad1;
    const float* dec1;      // 1 / W^(k)^2 per DFT bin of one axis (deconvolution), or NULL
    const float* ictab;
    double* pk_out;         // P(k): [slot][nbins] sums of w |delta^|^2
    int nbins;
    float scale;
    float kf;
};

enum { PM_Z_FORCE = 0, PM_Z_FORCE_IL = 1, PM_Z_IC = 2, PM_Z_PK = 3, PM_Z_ADJ = 4, PM_Z_IC_ADJ = 5, PM_Z_POT = 6,
       PM_Z_POT_IL = 7, PM_Z_IC_D2 = 8, PM_Z_IC_O2 = 9, PM_Z_LPT2 = 10, PM_Z_PKX = 11 };

// clear_in != 0: the input rows are zeroed after they are read (a density mesh
// consumed here is then ready for the next deposit without a separate memset)
int pm_fft_r2c_x(int log2n, const float* in, long long in_stride, float2* out, long long out_stride, int nmesh,
                 const float2* tw, cudaStream_t st, int clear_in = 0);
int pm_fft_c2r_x(int log2n, const float2* in, long long in_stride, float* out, long long out_stride, float* out2,
                 long long out2_stride, float scale2, int nmesh, const float2* tw, cudaStream_t st);
// inverse x pass of three spectra (comp_stride apart; slot q at q * slot_stride) into one
// interleaved float4 mesh (gx, gy, gz, 0) per q (out_stride float4 apart)
int pm_fft_c2r_x3(int log2n, const float2* in, long long comp_stride, long long slot_stride, float4* out,
                  long long out_stride, int nmesh, const float2* tw, cudaStream_t st);
int pm_fft_y(int log2n, float2* data, long long stride, int nmesh, int dir, const float2* tw, cudaStream_t st);
int pm_fft_z(int log2n, int mode, const PmZPass& p, int nslots, cudaStream_t st);

// force4[q][j] = (-D1_x phi, -D1_y phi, -D1_z phi, 0) at every cell of the n^3 mesh
// phi[q] (q < nmesh; phi slot stride phi_stride floats, force4 stride f_stride float4),
// D1 the finite-difference gradient of Table 2 of order 2, 4 or 6 (cell size 1/inv_h).
int pm_grad_stencil(int grad_order, int log2n, float inv_h, const float* phi, long long phi_stride, float4* force4,
                    long long f_stride, int nmesh, cudaStream_t st);

// div[q] = sum_c D1_c s_c of three planar meshes per q (c-th at c * n^3), the transpose
// partner of pm_grad_stencil.
int pm_div_stencil(int grad_order, int log2n, float inv_h, const float* s3, long long s_stride, float* div,
                   long long d_stride, int nmesh, cudaStream_t st);

// Particle kernels.  Geometry shared by deposit and interpolation.
struct PmGeom {
    int log2np;          // particles per dimension = 1 << log2np
    int log2ng;          // mesh cells per dimension = 1 << log2ng
    float inv_h;         // 1 / H, H = L / n_mesh
    long long slot_part; // floats between slots of one state component array (= 3 N)
    long long slot_mesh; // floats between slots of the mesh array passed (M per mesh x meshes per slot)
};

// rho[b] += sum_i W(r_j - X_i (+ shift)) for X = q + disp + tau1 * vel (vel may be null).
int pm_deposit(int order, const PmGeom& g, const float* disp, const float* vel, const SlotCoef* coef,
               int coef_stride, float shift_cells, float* rho, int nslots, cudaStream_t st);
// A = gather(g) / D_half^2 at X_half = q + disp + tau1 vel; V' = alpha V + kick A; disp' = disp + tau1 V + tau2 V'.
// force4: [slot][1 or 2 grids][M] float4 (gx, gy, gz, 0); the second grid is shifted by +1/2 cell.
// g.slot_mesh counts float4 per slot here.
// predrift_in: disp already holds X_half - q; coef_next (may be NULL): write X + (tau2 + tau1') V'.
int pm_interp_kick(int order, int interlace, const PmGeom& g, float* disp, float* vel, const SlotCoef* coef,
                   int coef_stride, const float4* force4, int nslots, cudaStream_t st, int predrift_in = 0,
                   const SlotCoef* coef_next = nullptr);
// acc[b][c][i] = sum_j g_c,j W(r_j - X_i) at X = q + disp (no kick): stage-level interpolation.
int pm_interp(int order, int interlace, const PmGeom& g, const float* disp, const float* force, float* acc,
              int nslots, cudaStream_t st);

// Adjoint (Sec. 2.7, Table 5; App. C pullbacks).  See particles.cu.
int pm_adj_drift_deposit(int order, const PmGeom& g, float* disp, const float* vel, const float* adisp, float* avel,
                         const SlotCoef* coef, int cstride, float* rho, int nslots, cudaStream_t st);
int pm_adj_interp(int order, const PmGeom& g, const float* disp, float* vel, float* adisp, const float* avel,
                  const SlotCoef* coef, int cstride, const float4* force4, float* s3, int nslots, cudaStream_t st);
int pm_adj_gather_grad(int order, int finish, const PmGeom& g, float* disp, const float* vel, float* adisp,
                       float* avel, const SlotCoef* coef, int cstride, const float* rhoa, float scale, int nslots,
                       cudaStream_t st);
int pm_dot(const float* a, const float* b, long long n, double* out, int nslots, cudaStream_t st);
int pm_axpby(float* out, const float* x, const float* y, float a, float b, long long n, cudaStream_t st);

// 2LPT source (Eq. LPT_kernels at n = 2) from three real fields t0..t2 of n elements
// per slot (slot stride 3n, mu slot stride n):
// pass 0 (diagonal psi_x,x, psi_y,y, psi_z,z): mu = t0 t1 + t0 t2 + t1 t2;
// pass 1 (off-diagonal psi_x,y, psi_x,z, psi_y,z): mu = -(3/7) (mu - t0^2 - t1^2 - t2^2) = L^(2).
int pm_lpt2_source(int pass, const float* t, float* mu, long long n, int nslots, cudaStream_t st);

// Forward mode (tangents of the DKD step).  drift = 1: X_half = X + tau1 V and its
// tangent (written back), then deposit X_half into rho (skipped when NULL) and
// rho' = sum X'_half . grad W into trho; drift = 0: deposit of X and X' as given.
int pm_jvp_drift_deposit(int order, int drift, const PmGeom& g, float* disp, const float* vel, float* tdisp,
                         const float* tvel, const SlotCoef* coef, int cstride, float* rho, float* trho, int nslots,
                         cudaStream_t st);
// A = gather(g), A' = gather(g') + X' . grad gather(g) at X = disp (= X_half); kick and
// drift_2 of the state and the tangent.
int pm_jvp_interp_kick(int order, const PmGeom& g, float* disp, float* vel, float* tdisp, float* tvel,
                       const SlotCoef* coef, int cstride, const float4* force4, const float4* tforce4, int nslots,
                       cudaStream_t st);
