// Particle <-> mesh kernels of the PM step:
//   deposit        (drift_1 of Eq. dkd fused with the mass assignment, Table 1)
//   interp + kick  (force interpolation with the same kernel, Sec. 2.5, fused with
//                   the kick and drift_2 of Eq. dkd)
// Positions are never formed in absolute coordinates: the cell index of a
// particle is its lattice index (integer) plus the floor of its displacement
// in cells, so float32 keeps full precision on the sub-cell fraction.
#include "pm_kernels.h"

namespace {

// Cell index (unwrapped) and sub-cell offset of lattice index il displaced by
// s cells, for a mesh 2^dshift times finer than the lattice (dshift may be < 0).
struct AxisTaps {
    int c;       // first tap cell (unwrapped)
    float w[3];  // weights of taps c, c+1 (CIC) or c, c+1, c+2 (TSC)
    float dw[3]; // d w / d u (u = position in cells), one-sided at CIC kinks as the floor gives
};

template <int ORDER>
__device__ __forceinline__ AxisTaps axis_taps(int il, int dshift, float s) {
    int base;
    float fr0;
    if (dshift >= 0) {
        base = il << dshift;
        fr0 = 0.f;
    } else {
        const int d = -dshift;
        base = il >> d;
        fr0 = (float)(il & ((1 << d) - 1)) * __int_as_float((127 - d) << 23);   // * 2^-d
    }
    const float t = fr0 + s;
    AxisTaps a;
    if (ORDER == 2) {
        // CIC (Table 1): cells floor(t), floor(t)+1, weights 1-f, f
        const float fl = floorf(t);
        const float f = t - fl;
        a.c = base + (int)fl;
        a.w[0] = 1.f - f;
        a.w[1] = f;
        a.w[2] = 0.f;
        a.dw[0] = -1.f;
        a.dw[1] = 1.f;
        a.dw[2] = 0.f;
    } else {
        // TSC (Table 1): nearest node i0 = floor(t + 1/2), d = t - i0 in [-1/2, 1/2)
        const float fl = floorf(t + 0.5f);
        const float d = t - fl;
        a.c = base + (int)fl - 1;
        a.w[0] = 0.5f * (0.5f - d) * (0.5f - d);
        a.w[1] = 0.75f - d * d;
        a.w[2] = 0.5f * (0.5f + d) * (0.5f + d);
        a.dw[0] = -(0.5f - d);
        a.dw[1] = -2.f * d;
        a.dw[2] = 0.5f + d;
    }
    return a;
}

struct Lattice {
    int ix, iy, iz;
};

__device__ __forceinline__ Lattice lattice_index(long long i, int log2np) {
    const int m = (1 << log2np) - 1;
    Lattice l;
    l.ix = (int)(i & m);
    l.iy = (int)((i >> log2np) & m);
    l.iz = (int)(i >> (2 * log2np));
    return l;
}

template <int ORDER>
__global__ void __launch_bounds__(256) k_deposit(PmGeom g, const float* __restrict__ disp,
                                                 const float* __restrict__ vel, const SlotCoef* __restrict__ coef,
                                                 int cstride, float shift, float* __restrict__ rho) {
    const int slot = blockIdx.y;
    const SlotCoef cf = coef[slot * cstride];
    if (!cf.active) return;
    const long long N = 1ll << (3 * g.log2np);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Lattice L = lattice_index(i, g.log2np);
    const float* d = disp + slot * g.slot_part;
    float sx = d[i], sy = d[N + i], sz = d[2 * N + i];
    if (vel) {
        const float* v = vel + slot * g.slot_part;
        sx += cf.tau1 * v[i];
        sy += cf.tau1 * v[N + i];
        sz += cf.tau1 * v[2 * N + i];
    }
    const int ds = g.log2ng - g.log2np;
    const AxisTaps ax = axis_taps<ORDER>(L.ix, ds, sx * g.inv_h + shift);
    const AxisTaps ay = axis_taps<ORDER>(L.iy, ds, sy * g.inv_h + shift);
    const AxisTaps az = axis_taps<ORDER>(L.iz, ds, sz * g.inv_h + shift);
    const int ng = 1 << g.log2ng, msk = ng - 1;
    float* m = rho + slot * g.slot_mesh;
#pragma unroll
    for (int c = 0; c < ORDER; ++c) {
        const long long zo = (long long)((az.c + c) & msk) * ng;
#pragma unroll
        for (int b = 0; b < ORDER; ++b) {
            const long long yo = (zo + ((ay.c + b) & msk)) * ng;
            const float wzy = az.w[c] * ay.w[b];
#pragma unroll
            for (int a = 0; a < ORDER; ++a) atomicAdd(&m[yo + ((ax.c + a) & msk)], wzy * ax.w[a]);
        }
    }
}

// sum over taps of g_c at the particle, c = 0..2, meshes at f, f + M, f + 2M
template <int ORDER>
__device__ __forceinline__ void gather3(const float* __restrict__ f, long long M, int log2ng, const AxisTaps& ax,
                                        const AxisTaps& ay, const AxisTaps& az, float acc[3]) {
    const int ng = 1 << log2ng, msk = ng - 1;
#pragma unroll
    for (int c = 0; c < ORDER; ++c) {
        const long long zo = (long long)((az.c + c) & msk) * ng;
#pragma unroll
        for (int b = 0; b < ORDER; ++b) {
            const long long yo = (zo + ((ay.c + b) & msk)) * ng;
            const float wzy = az.w[c] * ay.w[b];
#pragma unroll
            for (int a = 0; a < ORDER; ++a) {
                const long long j = yo + ((ax.c + a) & msk);
                const float w = wzy * ax.w[a];
                acc[0] += w * __ldg(&f[j]);
                acc[1] += w * __ldg(&f[M + j]);
                acc[2] += w * __ldg(&f[2 * M + j]);
            }
        }
    }
}

template <int ORDER, int IL, int KICK>
__global__ void __launch_bounds__(256) k_interp(PmGeom g, float* __restrict__ disp, float* __restrict__ vel,
                                                const SlotCoef* __restrict__ coef, int cstride,
                                                const float* __restrict__ force, float* __restrict__ acc_out) {
    const int slot = blockIdx.y;
    SlotCoef cf;
    if (KICK) {
        cf = coef[slot * cstride];
        if (!cf.active) return;
    }
    const long long N = 1ll << (3 * g.log2np);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Lattice L = lattice_index(i, g.log2np);
    float* d = disp + slot * g.slot_part;
    float* v = vel + slot * g.slot_part;
    float p[3] = {d[i], d[N + i], d[2 * N + i]};
    float u[3];
    if (KICK) {
        u[0] = v[i];
        u[1] = v[N + i];
        u[2] = v[2 * N + i];
#pragma unroll
        for (int c = 0; c < 3; ++c) p[c] += cf.tau1 * u[c];    // drift_1: X_half
    }
    const int ds = g.log2ng - g.log2np;
    const long long M = 1ll << (3 * g.log2ng);
    const float* f = force + slot * g.slot_mesh;    // slot_mesh = (3 or 6) * M here
    float acc[3] = {0.f, 0.f, 0.f};
    {
        const AxisTaps ax = axis_taps<ORDER>(L.ix, ds, p[0] * g.inv_h);
        const AxisTaps ay = axis_taps<ORDER>(L.iy, ds, p[1] * g.inv_h);
        const AxisTaps az = axis_taps<ORDER>(L.iz, ds, p[2] * g.inv_h);
        gather3<ORDER>(f, M, g.log2ng, ax, ay, az, acc);
    }
    if (IL) {
        // second grid shifted by half a cell; average the two interpolants
        float acc1[3] = {0.f, 0.f, 0.f};
        const AxisTaps ax = axis_taps<ORDER>(L.ix, ds, p[0] * g.inv_h + 0.5f);
        const AxisTaps ay = axis_taps<ORDER>(L.iy, ds, p[1] * g.inv_h + 0.5f);
        const AxisTaps az = axis_taps<ORDER>(L.iz, ds, p[2] * g.inv_h + 0.5f);
        gather3<ORDER>(f + 3 * M, M, g.log2ng, ax, ay, az, acc1);
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = 0.5f * (acc[c] + acc1[c]);
    }
    if (KICK) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float vn = cf.alpha * u[c] + cf.kick * acc[c];   // kick
            v[c * N + i] = vn;
            d[c * N + i] = p[c] + cf.tau2 * vn;                     // drift_2
        }
    } else {
        float* o = acc_out + slot * g.slot_part;
#pragma unroll
        for (int c = 0; c < 3; ++c) o[c * N + i] = acc[c];
    }
}

// ------------------------------------------------------------------ adjoint
// Backward-in-time DKD (Sec. 2.7, Table 5) with the App. C pullbacks of the
// scatter (deposit) and gather (interpolation).  g = G rho with
// G_c = (1/N) IDFT diag(m_c) DFT, A = g / D_half^2, kick = beta / D_half^2.

// primal drift back X_half = X - tau2 V, adjoint drift V* += tau2 X*, then the
// deposit of X_half (mesh rho) for the force recomputation
template <int ORDER>
__global__ void __launch_bounds__(256) k_adj_drift_deposit(PmGeom g, float* __restrict__ disp,
                                                           const float* __restrict__ vel,
                                                           const float* __restrict__ adisp, float* __restrict__ avel,
                                                           const SlotCoef* __restrict__ coef, int cstride,
                                                           float* __restrict__ rho) {
    const int slot = blockIdx.y;
    const SlotCoef cf = coef[slot * cstride];
    if (!cf.active) return;
    const long long N = 1ll << (3 * g.log2np);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Lattice L = lattice_index(i, g.log2np);
    const long long o = slot * g.slot_part;
    float p[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        p[c] = disp[o + c * N + i] - cf.tau2 * vel[o + c * N + i];
        disp[o + c * N + i] = p[c];
        avel[o + c * N + i] += cf.tau2 * adisp[o + c * N + i];
    }
    const int ds = g.log2ng - g.log2np;
    const AxisTaps ax = axis_taps<ORDER>(L.ix, ds, p[0] * g.inv_h);
    const AxisTaps ay = axis_taps<ORDER>(L.iy, ds, p[1] * g.inv_h);
    const AxisTaps az = axis_taps<ORDER>(L.iz, ds, p[2] * g.inv_h);
    const int ng = 1 << g.log2ng, msk = ng - 1;
    float* m = rho + slot * g.slot_mesh;
#pragma unroll
    for (int c = 0; c < ORDER; ++c) {
        const long long zo = (long long)((az.c + c) & msk) * ng;
#pragma unroll
        for (int b = 0; b < ORDER; ++b) {
            const long long yo = (zo + ((ay.c + b) & msk)) * ng;
            const float wzy = az.w[c] * ay.w[b];
#pragma unroll
            for (int a = 0; a < ORDER; ++a) atomicAdd(&m[yo + ((ax.c + a) & msk)], wzy * ax.w[a]);
        }
    }
}

// At X_half: A = gather(g); V_prev = (V - kick A) / alpha;
// X* += kick sum_c u_c grad gather(g_c) with u = V* (adjoint kick, gather term);
// s_c += u_c W (the mesh cotangent of the gather, a 3-channel scatter).
template <int ORDER>
__global__ void __launch_bounds__(256) k_adj_interp(PmGeom g, const float* __restrict__ disp, float* __restrict__ vel,
                                                    float* __restrict__ adisp, const float* __restrict__ avel,
                                                    const SlotCoef* __restrict__ coef, int cstride,
                                                    const float* __restrict__ force, float* __restrict__ s3) {
    const int slot = blockIdx.y;
    const SlotCoef cf = coef[slot * cstride];
    if (!cf.active) return;
    const long long N = 1ll << (3 * g.log2np);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Lattice L = lattice_index(i, g.log2np);
    const long long o = slot * g.slot_part;
    float p[3], u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        p[c] = disp[o + c * N + i];
        u[c] = avel[o + c * N + i];
    }
    const int ds = g.log2ng - g.log2np;
    const AxisTaps ax = axis_taps<ORDER>(L.ix, ds, p[0] * g.inv_h);
    const AxisTaps ay = axis_taps<ORDER>(L.iy, ds, p[1] * g.inv_h);
    const AxisTaps az = axis_taps<ORDER>(L.iz, ds, p[2] * g.inv_h);
    const int ng = 1 << g.log2ng, msk = ng - 1;
    const long long M = 1ll << (3 * g.log2ng);
    const float* f = force + slot * 3 * M;
    float* sm = s3 + slot * 3 * M;
    float A[3] = {0.f, 0.f, 0.f};
    float t[3] = {0.f, 0.f, 0.f};   // sum_c u_c d/du_d gather(g_c)
#pragma unroll
    for (int c = 0; c < ORDER; ++c) {
        const long long zo = (long long)((az.c + c) & msk) * ng;
#pragma unroll
        for (int b = 0; b < ORDER; ++b) {
            const long long yo = (zo + ((ay.c + b) & msk)) * ng;
#pragma unroll
            for (int a = 0; a < ORDER; ++a) {
                const long long j = yo + ((ax.c + a) & msk);
                const float w = az.w[c] * ay.w[b] * ax.w[a];
                const float g0 = __ldg(&f[j]), g1 = __ldg(&f[M + j]), g2 = __ldg(&f[2 * M + j]);
                A[0] += w * g0;
                A[1] += w * g1;
                A[2] += w * g2;
                const float ug = u[0] * g0 + u[1] * g1 + u[2] * g2;
                t[0] += ug * ax.dw[a] * ay.w[b] * az.w[c];
                t[1] += ug * ax.w[a] * ay.dw[b] * az.w[c];
                t[2] += ug * ax.w[a] * ay.w[b] * az.dw[c];
                atomicAdd(&sm[j], u[0] * w);
                atomicAdd(&sm[M + j], u[1] * w);
                atomicAdd(&sm[2 * M + j], u[2] * w);
            }
        }
    }
    const float ia = 1.f / cf.alpha;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        vel[o + c * N + i] = (vel[o + c * N + i] - cf.kick * A[c]) * ia;          // primal kick back
        adisp[o + c * N + i] += cf.kick * g.inv_h * t[c];                          // d/dX = inv_h d/du
    }
}

// X* += kick grad gather(rho*) (scatter pullback w.r.t. positions);
// V* <- alpha V*; X <- X_half - tau1 V_prev; V* += tau1 X*.
// With FINISH = 0: out = scale * grad gather(rho*) at X = q + disp only (density VJP).
template <int ORDER, int FINISH>
__global__ void __launch_bounds__(256) k_adj_gather_grad(PmGeom g, float* __restrict__ disp,
                                                         const float* __restrict__ vel, float* __restrict__ adisp,
                                                         float* __restrict__ avel, const SlotCoef* __restrict__ coef,
                                                         int cstride, const float* __restrict__ rhoa, float scale) {
    const int slot = blockIdx.y;
    SlotCoef cf{};
    if (FINISH) {
        cf = coef[slot * cstride];
        if (!cf.active) return;
    }
    const long long N = 1ll << (3 * g.log2np);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Lattice L = lattice_index(i, g.log2np);
    const long long o = slot * g.slot_part;
    float p[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) p[c] = disp[o + c * N + i];
    const int ds = g.log2ng - g.log2np;
    const AxisTaps ax = axis_taps<ORDER>(L.ix, ds, p[0] * g.inv_h);
    const AxisTaps ay = axis_taps<ORDER>(L.iy, ds, p[1] * g.inv_h);
    const AxisTaps az = axis_taps<ORDER>(L.iz, ds, p[2] * g.inv_h);
    const int ng = 1 << g.log2ng, msk = ng - 1;
    const float* r = rhoa + slot * g.slot_mesh;
    float t[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < ORDER; ++c) {
        const long long zo = (long long)((az.c + c) & msk) * ng;
#pragma unroll
        for (int b = 0; b < ORDER; ++b) {
            const long long yo = (zo + ((ay.c + b) & msk)) * ng;
#pragma unroll
            for (int a = 0; a < ORDER; ++a) {
                const float rv = __ldg(&r[yo + ((ax.c + a) & msk)]);
                t[0] += rv * ax.dw[a] * ay.w[b] * az.w[c];
                t[1] += rv * ax.w[a] * ay.dw[b] * az.w[c];
                t[2] += rv * ax.w[a] * ay.w[b] * az.dw[c];
            }
        }
    }
    if (FINISH) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float xa = adisp[o + c * N + i] + cf.kick * g.inv_h * t[c];
            adisp[o + c * N + i] = xa;
            avel[o + c * N + i] = cf.alpha * avel[o + c * N + i] + cf.tau1 * xa;
            disp[o + c * N + i] = p[c] - cf.tau1 * vel[o + c * N + i];
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) adisp[o + c * N + i] = scale * g.inv_h * t[c];
    }
}

// per-slot FP64 dot products sum_i a_i b_i over n floats (slot stride n)
__global__ void __launch_bounds__(256) k_dot(const float* __restrict__ a, const float* __restrict__ b, long long n,
                                            double* __restrict__ out) {
    const int slot = blockIdx.y;
    const float* x = a + slot * n;
    const float* y = b + slot * n;
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += (double)x[i] * (double)y[i];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&out[slot], red[0]);
}

// out = a * x + b * y elementwise
__global__ void k_axpby(float* __restrict__ out, const float* __restrict__ x, const float* __restrict__ y, float a,
                        float b, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + b * y[i];
}

}  // namespace

int pm_deposit(int order, const PmGeom& g, const float* disp, const float* vel, const SlotCoef* coef, int coef_stride,
               float shift_cells, float* rho, int nslots, cudaStream_t st) {
    const long long N = 1ll << (3 * g.log2np);
    dim3 grid((unsigned)((N + 255) / 256), nslots);
    if (order == 2)
        k_deposit<2><<<grid, 256, 0, st>>>(g, disp, vel, coef, coef_stride, shift_cells, rho);
    else if (order == 3)
        k_deposit<3><<<grid, 256, 0, st>>>(g, disp, vel, coef, coef_stride, shift_cells, rho);
    else
        return -1;
    return 0;
}

int pm_interp_kick(int order, int interlace, const PmGeom& g, float* disp, float* vel, const SlotCoef* coef,
                   int coef_stride, const float* force, int nslots, cudaStream_t st) {
    const long long N = 1ll << (3 * g.log2np);
    dim3 grid((unsigned)((N + 255) / 256), nslots);
#define PM_IK(O, I) k_interp<O, I, 1><<<grid, 256, 0, st>>>(g, disp, vel, coef, coef_stride, force, nullptr)
    if (order == 2 && !interlace) PM_IK(2, 0);
    else if (order == 2 && interlace) PM_IK(2, 1);
    else if (order == 3 && !interlace) PM_IK(3, 0);
    else if (order == 3 && interlace) PM_IK(3, 1);
    else return -1;
#undef PM_IK
    return 0;
}

int pm_interp(int order, int interlace, const PmGeom& g, const float* disp, const float* force, float* acc,
              int nslots, cudaStream_t st) {
    const long long N = 1ll << (3 * g.log2np);
    dim3 grid((unsigned)((N + 255) / 256), nslots);
    float* d = const_cast<float*>(disp);
#define PM_I(O, I) k_interp<O, I, 0><<<grid, 256, 0, st>>>(g, d, nullptr, nullptr, 0, force, acc)
    if (order == 2 && !interlace) PM_I(2, 0);
    else if (order == 2 && interlace) PM_I(2, 1);
    else if (order == 3 && !interlace) PM_I(3, 0);
    else if (order == 3 && interlace) PM_I(3, 1);
    else return -1;
#undef PM_I
    return 0;
}

int pm_adj_drift_deposit(int order, const PmGeom& g, float* disp, const float* vel, const float* adisp, float* avel,
                         const SlotCoef* coef, int cstride, float* rho, int nslots, cudaStream_t st) {
    const long long N = 1ll << (3 * g.log2np);
    dim3 grid((unsigned)((N + 255) / 256), nslots);
    if (order == 2) k_adj_drift_deposit<2><<<grid, 256, 0, st>>>(g, disp, vel, adisp, avel, coef, cstride, rho);
    else if (order == 3) k_adj_drift_deposit<3><<<grid, 256, 0, st>>>(g, disp, vel, adisp, avel, coef, cstride, rho);
    else return -1;
    return 0;
}

int pm_adj_interp(int order, const PmGeom& g, const float* disp, float* vel, float* adisp, const float* avel,
                  const SlotCoef* coef, int cstride, const float* force, float* s3, int nslots, cudaStream_t st) {
    const long long N = 1ll << (3 * g.log2np);
    dim3 grid((unsigned)((N + 255) / 256), nslots);
    if (order == 2) k_adj_interp<2><<<grid, 256, 0, st>>>(g, disp, vel, adisp, avel, coef, cstride, force, s3);
    else if (order == 3) k_adj_interp<3><<<grid, 256, 0, st>>>(g, disp, vel, adisp, avel, coef, cstride, force, s3);
    else return -1;
    return 0;
}

int pm_adj_gather_grad(int order, int finish, const PmGeom& g, float* disp, const float* vel, float* adisp,
                       float* avel, const SlotCoef* coef, int cstride, const float* rhoa, float scale, int nslots,
                       cudaStream_t st) {
    const long long N = 1ll << (3 * g.log2np);
    dim3 grid((unsigned)((N + 255) / 256), nslots);
#define PM_AG(O, F) k_adj_gather_grad<O, F><<<grid, 256, 0, st>>>(g, disp, vel, adisp, avel, coef, cstride, rhoa, scale)
    if (order == 2 && finish) PM_AG(2, 1);
    else if (order == 2) PM_AG(2, 0);
    else if (order == 3 && finish) PM_AG(3, 1);
    else if (order == 3) PM_AG(3, 0);
    else return -1;
#undef PM_AG
    return 0;
}

int pm_dot(const float* a, const float* b, long long n, double* out, int nslots, cudaStream_t st) {
    dim3 grid(304, nslots);
    k_dot<<<grid, 256, 0, st>>>(a, b, n, out);
    return 0;
}

int pm_axpby(float* out, const float* x, const float* y, float a, float b, long long n, cudaStream_t st) {
    k_axpby<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, x, y, a, b, n);
    return 0;
}
