// Shared device-side definitions for the PM (particle-mesh) kernels.
//
// Layouts (all device memory, all float32 unless noted):
//   particle state  disp[b][c][i], vel[b][c][i]   slot b, component c = x,y,z,
//                   particle i = (iz*np + iy)*np + ix on the Lagrangian lattice
//                   q = (ix, iy, iz) * L / np; disp = X - q (Sec. 2.2 displacement).
//   real mesh       rho[b][z][y][x], n^3 per slot, node j at r_j = j*H, H = L/n.
//   half spectrum   spec[b][z][y][kx], row pitch P = n/2 + SPEC_PAD complex, valid
//                   kx in [0, n/2]; the columns past n/2 are padding that the
//                   column passes read and write but nothing else uses.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define SPEC_PAD 8          // complex padding per spectrum row (= column tile width)
#define COL_TILE 8          // kx columns per CTA in the y / z passes

struct SlotCoef {           // per-slot kick/drift coefficients for one DKD step (Eq. dkd)
    float tau1, tau2, alpha, kick;  // kick = beta / D_half^2 (A = g / D_half^2)
    int   active;                   // 0: slot idle, kernels leave it untouched
    int   pad[3];
};

__host__ __device__ inline int spec_pitch(int n) { return n / 2 + SPEC_PAD; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by +i (dir > 0) or -i (dir < 0)
__device__ __forceinline__ float2 cmul_i(float2 a, int dir) {
    return dir > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Wavenumber index m in [-n/2, n/2) of DFT bin j (bin n/2 taken as -n/2, the Nyquist mode).
__device__ __forceinline__ int freq_index(int j, int n) { return j < n / 2 ? j : j - n; }
