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
    float w[5];  // weights of taps c, c+1 (CIC), c .. c+2 (TSC), c .. c+3 (PCS) or c .. c+4 (ES, NUFFT)
    float dw[5]; // d w / d u (u = position in cells), one-sided at CIC kinks as the floor gives
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
    } else if (ORDER == 5) {
        // ES kernel of the NUFFT force (width 5, beta = 2.3 * 5): nearest node i0 =
        // floor(t + 1/2), taps i0-2 .. i0+2, weight exp(beta (sqrt(1 - z^2) - 1)) with
        // z = 2 x / 5 at distance x = cell - t (no derivatives: forward only)
        const float fl = floorf(t + 0.5f);
        a.c = base + (int)fl - 2;
#pragma unroll
        for (int o = 0; o < 5; ++o) {
            const float z = 0.4f * (fl + (float)(o - 2) - t);
            const float r = 1.f - z * z;
            a.w[o] = r >= 0.f ? expf(11.5f * (sqrtf(r) - 1.f)) : 0.f;
            a.dw[o] = 0.f;
        }
        return a;
    } else if (ORDER == 4) {
        // PCS (Table 1, cubic B-spline): cells floor(t)-1 .. floor(t)+2 at distances
        // 1+d, d, 1-d, 2-d (d = t - floor(t)); dw/du = -W'(x) at x = cell - u
        const float fl = floorf(t);
        const float d = t - fl, e = 1.f - d;
        a.c = base + (int)fl - 1;
        a.w[0] = e * e * e * (1.f / 6.f);
        a.w[1] = (4.f - 6.f * d * d + 3.f * d * d * d) * (1.f / 6.f);
        a.w[2] = (4.f - 6.f * e * e + 3.f * e * e * e) * (1.f / 6.f);
        a.w[3] = d * d * d * (1.f / 6.f);
        a.dw[0] = -0.5f * e * e;
        a.dw[1] = -2.f * d + 1.5f * d * d;
        a.dw[2] = 2.f * e - 1.5f * e * e;
        a.dw[3] = 0.5f * d * d;
        return a;
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

// L2 prefetch of the 128-byte line holding p (no registers held, nothing returned)
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// particles ahead of the current ones whose state lines each warp prefetches into L2:
// about the number of particles resident on the GPU at once, so that their state
// arrives while the current ones wait on their force gathers
constexpr long long STATE_PREFETCH = 1ll << 17;

// same from an interleaved float4 mesh (gx, gy, gz, 0): one 16-byte load per tap.
// Offsets are 32-bit (meshes hold at most 2^30 cells) and the periodic wrap of
// each axis is taken once per tap line, not per tap.
template <int ORDER>
__device__ __forceinline__ void gather3v(const float4* __restrict__ f, int log2ng, const AxisTaps& ax,
                                         const AxisTaps& ay, const AxisTaps& az, float acc[3]) {
    const int msk = (1 << log2ng) - 1;
    int xo[ORDER], yo[ORDER], zo[ORDER];
#pragma unroll
    for (int a = 0; a < ORDER; ++a) {
        xo[a] = (ax.c + a) & msk;
        yo[a] = ((ay.c + a) & msk) << log2ng;
        zo[a] = ((az.c + a) & msk) << (2 * log2ng);
    }
#pragma unroll
    for (int c = 0; c < ORDER; ++c) {
#pragma unroll
        for (int b = 0; b < ORDER; ++b) {
            const int row = zo[c] + yo[b];
            const float wzy = az.w[c] * ay.w[b];
#pragma unroll
            for (int a = 0; a < ORDER; ++a) {
                const float4 v = __ldg(f + (row + xo[a]));
                const float w = wzy * ax.w[a];
                acc[0] += w * v.x;
                acc[1] += w * v.y;
                acc[2] += w * v.z;
            }
        }
    }
}

// Lagrangian-tile deposit through a shared-memory window.
// A tile is (32/R) x (8/R) x (8/R) lattice sites (R = n_mesh / n_part in {1, 2}),
// i.e. a 32 x 8 x 8 block of cells before the particles move.  Its window is
// WX x WY x WZ cells: that block shifted by the tile's rounded mean displacement
// and padded by DEP_HALO cells (the x origin aligned down to 4 cells, so that
// every group of 4 cells is 16-byte aligned and never straddles the periodic
// boundary).  Each particle adds its ORDER^3 weights with shared-memory atomics
// (particles whose taps leave the window add straight to global memory), and
// the window is flushed with one 16-byte vector reduction per non-zero group.
// The window accumulates in unsigned fixed point, weight * 2^20 rounded: integer
// shared-memory atomics are native (float ones are not), the sums are exact and
// order-independent, and a cell cannot overflow since at most 2048 particles
// (one tile) add at most 2^20 each.
constexpr int DEP_HALO = 3;
constexpr float DEP_FIX = 1048576.f;            // 2^20
constexpr float DEP_UNFIX = 1.f / 1048576.f;

template <int ORDER>
struct DepWindow {
    static constexpr int LO = ORDER == 5 ? 2 : (ORDER >= 3 ? 1 : 0);   // taps below the base cell
    static constexpr int HALO = ORDER >= 4 ? 2 : DEP_HALO;   // PCS (4 taps) and ES (5) leave room for 2
    static constexpr int WX = 64;                   // >= 32 + 2 halo + ORDER - 1 + alignment slack; a multiple of 32
    static constexpr int WY = 16;                   // 8 + 2 halo + ORDER - 1, rounded up
    static constexpr int WZ = 16;
    static constexpr int QX = WX / 4;               // 16-byte groups per window row
    static constexpr int CELLS = WX * WY * WZ;
    static_assert(QX <= 16 && WY == 16, "flush maps 16 lanes per row, 16 rows per plane");
    static_assert(32 + 2 * HALO + ORDER - 1 + 3 <= WX && 8 + 2 * HALO + ORDER - 1 <= WY, "window");
};

__device__ __forceinline__ void red_v4(float* p, float4 v) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w)
                 : "memory");
}

// Tile geometry of the Lagrangian-tile kernels (R = n_mesh / n_part in {1, 2}).
// Thread t holds the particles p = 0..PPT-1 at x = ix0 + t % TXP and rows
// (t / TXP + RSTEP p) of the tile's TYP x TZP lattice rows; RSTEP is a multiple
// of TYP, so particle p sits p * RSTEP / TYP lattice planes above particle 0.
template <int R>
struct TileGeom {
    static constexpr int TXP = 32 / R, TYP = 8 / R, TZP = 8 / R;
    static constexpr int PPT = TXP * TYP * TZP / 256;    // particles per thread
    static constexpr int RSTEP = 256 / TXP;               // rows advanced per particle slot
    static constexpr int DZ = RSTEP / TYP;                // planes advanced per particle slot
    static_assert(RSTEP % TYP == 0, "tile rows");
    int ix0, iy0, iz0;   // tile origin (lattice)
    int ix, iy, iz;      // this thread's particle 0 (lattice)
    __device__ TileGeom(int tile, int log2np) {
        constexpr int LX = R == 2 ? 4 : 5, LY = R == 2 ? 2 : 3;   // log2 TXP, log2 TYP (= log2 TZP)
        const int lnx = log2np - LX, lny = log2np - LY;            // log2 of the tile counts along x, y
        ix0 = (tile & ((1 << lnx) - 1)) << LX;
        iy0 = ((tile >> lnx) & ((1 << lny) - 1)) << LY;
        iz0 = (tile >> (lnx + lny)) << LY;
        const int r = threadIdx.x / TXP;
        ix = ix0 + threadIdx.x % TXP;
        iy = iy0 + r % TYP;
        iz = iz0 + r / TYP;
    }
};

// Persistent tile deposit: CTA b walks tiles b, b + gridDim.x, ...  Per tile the
// drifted displacements (in cells) are loaded while the next tile's state lines
// are prefetched into L2, block-reduced to their mean (which places the window),
// scattered into the window, and the window is flushed.  The flush clears every
// group it adds to the mesh, so the window is all-zero again for the next tile
// with no separate clearing pass; the barrier after the first reduction of the
// next tile orders that clearing before the next atomics.
template <int ORDER, int R>
__global__ void __launch_bounds__(256, 4) k_deposit_tiled(PmGeom g, const float* __restrict__ disp,
                                                          const float* __restrict__ vel,
                                                          const SlotCoef* __restrict__ coef, int cstride,
                                                          float shift, float* __restrict__ rho, int ntiles) {
    using Win = DepWindow<ORDER>;
    using TG = TileGeom<R>;
    constexpr int PPT = TG::PPT;
    constexpr int DS = R == 2 ? 1 : 0;                    // log2 R
    extern __shared__ uint4 win4[];
    unsigned* win = reinterpret_cast<unsigned*>(win4);
    __shared__ __align__(16) float red[3][8];
    const int slot = blockIdx.y;
    const SlotCoef cf = coef[slot * cstride];
    if (!cf.active) return;
    const int t = threadIdx.x;
    const int np = 1 << g.log2np;
    const long long N = 1ll << (3 * g.log2np);
    const float* dx = disp + slot * g.slot_part;
    const float* dy = dx + N;
    const float* dz = dy + N;
    const float* vx = vel ? vel + slot * g.slot_part : nullptr;
    float* m = rho + slot * g.slot_mesh;
    const int log2ng = g.log2ng, ng = 1 << log2ng, msk = ng - 1;
    const int plane = np * np;                            // lattice sites per plane (< 2^31)
    for (int i = t; i < Win::CELLS / 4; i += 256) win4[i] = make_uint4(0u, 0u, 0u, 0u);
    // flush geometry of this thread: group q of row y in every plane
    const int fq = t & 15, fy = t >> 4;

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const TG T(tile, g.log2np);
        if (tile + (int)gridDim.x < ntiles && t < 3 * TG::TYP * TG::TZP) {
            // L2 prefetch of the next tile's lattice rows (component, row) of disp (and vel)
            const TG Tn(tile + gridDim.x, g.log2np);
            const int c = t / (TG::TYP * TG::TZP), row = t % (TG::TYP * TG::TZP);
            const long long i0 = c * N + ((long long)(Tn.iz0 + row / TG::TYP) * np + Tn.iy0 + row % TG::TYP) * np + Tn.ix0;
            prefetch_l2(dx + i0);
            if (vx) prefetch_l2(vx + i0);
        }
        const int i0 = (T.iz * np + T.iy) * np + T.ix;    // particle 0 of this thread
        float sx[PPT], sy[PPT], sz[PPT];
        float m0 = 0.f, m1 = 0.f, m2 = 0.f;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const int i = i0 + p * TG::DZ * plane;
            float a = dx[i], b = dy[i], c = dz[i];
            if (vx) {
                a += cf.tau1 * vx[i];
                b += cf.tau1 * vx[N + i];
                c += cf.tau1 * vx[2 * N + i];
            }
            sx[p] = a * g.inv_h + shift;
            sy[p] = b * g.inv_h + shift;
            sz[p] = c * g.inv_h + shift;
            m0 += sx[p];
            m1 += sy[p];
            m2 += sz[p];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m0 += __shfl_xor_sync(0xffffffffu, m0, o);
            m1 += __shfl_xor_sync(0xffffffffu, m1, o);
            m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        }
        if ((t & 31) == 0) {
            red[0][t >> 5] = m0;
            red[1][t >> 5] = m1;
            red[2][t >> 5] = m2;
        }
        __syncthreads();
        float mean[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float4 u = reinterpret_cast<const float4*>(red[c])[0];
            const float4 w = reinterpret_cast<const float4*>(red[c])[1];
            mean[c] = ((u.x + u.y) + (u.z + u.w) + ((w.x + w.y) + (w.z + w.w))) *
                      (1.f / (TG::TXP * TG::TYP * TG::TZP));
        }
        const int ox = (T.ix0 * R + __float2int_rn(mean[0]) - Win::HALO - Win::LO) & ~3;
        const int oy = T.iy0 * R + __float2int_rn(mean[1]) - Win::HALO - Win::LO;
        const int oz = T.iz0 * R + __float2int_rn(mean[2]) - Win::HALO - Win::LO;
#pragma unroll
        for (int p = 0; p < PPT; ++p) {
            const AxisTaps ax = axis_taps<ORDER>(T.ix, DS, sx[p]);
            const AxisTaps ay = axis_taps<ORDER>(T.iy, DS, sy[p]);
            const AxisTaps az = axis_taps<ORDER>(T.iz + p * TG::DZ, DS, sz[p]);
            const int lx = ax.c - ox, ly = ay.c - oy, lz = az.c - oz;
            const bool inside = (unsigned)lx <= (unsigned)(Win::WX - ORDER) &&
                                (unsigned)ly <= (unsigned)(Win::WY - ORDER) &&
                                (unsigned)lz <= (unsigned)(Win::WZ - ORDER);
            if (inside) {
                unsigned* w0 = win + (lz * Win::WY + ly) * Win::WX + lx;
#pragma unroll
                for (int c = 0; c < ORDER; ++c) {
                    const float wz = az.w[c] * DEP_FIX;
#pragma unroll
                    for (int b = 0; b < ORDER; ++b) {
                        const float wzy = wz * ay.w[b];
#pragma unroll
                        for (int a = 0; a < ORDER; ++a)
                            atomicAdd(w0 + (c * Win::WY + b) * Win::WX + a, __float2uint_rn(wzy * ax.w[a]));
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < ORDER; ++c) {
                    const long long zo = (long long)((az.c + c) & msk) << log2ng;
#pragma unroll
                    for (int b = 0; b < ORDER; ++b) {
                        const long long yo = (zo + ((ay.c + b) & msk)) << log2ng;
                        const float wzy = az.w[c] * ay.w[b];
#pragma unroll
                        for (int a = 0; a < ORDER; ++a) atomicAdd(&m[yo + ((ax.c + a) & msk)], wzy * ax.w[a]);
                    }
                }
            }
        }
        __syncthreads();
        // flush: this thread's group fq of row fy in each of the WZ planes; clear what it adds
        if (fq < Win::QX) {
            const int row = (((oy + fy) & msk) << log2ng) + ((ox + 4 * fq) & msk);
            uint4* src = win4 + fy * Win::QX + fq;
#pragma unroll 4
            for (int z = 0; z < Win::WZ; ++z) {
                const uint4 u = src[z * Win::WY * Win::QX];
                if ((u.x | u.y | u.z | u.w) != 0u) {
                    src[z * Win::WY * Win::QX] = make_uint4(0u, 0u, 0u, 0u);
                    const float4 val =
                        make_float4(u.x * DEP_UNFIX, u.y * DEP_UNFIX, u.z * DEP_UNFIX, u.w * DEP_UNFIX);
                    red_v4(m + ((long long)((oz + z) & msk) << (2 * log2ng)) + row, val);
                }
            }
        }
    }
}

// interpolation + kick + drift_2 from interleaved float4 force meshes [slot][grid][M].
// Each thread handles IK_PPT particles 256 apart, so that the state loads and the
// gathers of several particles are in flight at once (the kernel is bound by the
// latency of its dependent loads: state -> cell -> force taps).
// Inside a multi-step run the positions between steps can be carried already
// drifted by the next step's tau1 (so the next deposit reads positions only):
// predrift_in = the input disp already holds X_half - q; coef_next != NULL = write
// X_half' - q = X + (tau2 + tau1') V' instead of X' - q.
constexpr int IK_PPT = 2;

// particles per thread of k_interp_kick: one for the wide kernels (PCS, ES)
__host__ __device__ constexpr int ik_ppt(int order) { return order >= 4 ? 1 : IK_PPT; }

template <int ORDER, int IL>
__global__ void __launch_bounds__(256) k_interp_kick(PmGeom g, float* __restrict__ disp, float* __restrict__ vel,
                                                     const SlotCoef* __restrict__ coef, int cstride,
                                                     const float4* __restrict__ force4, int predrift_in,
                                                     const SlotCoef* __restrict__ coef_next) {
    const int slot = blockIdx.y;
    const SlotCoef cf = coef[slot * cstride];
    if (!cf.active) return;
    const float tin = predrift_in ? 0.f : cf.tau1;
    const float tout = cf.tau2 + (coef_next ? coef_next[slot * cstride].tau1 : 0.f);
    const int N = 1 << (3 * g.log2np);                  // at most 2^30 particles per slot
    constexpr int PPT = ik_ppt(ORDER);
    const int i0 = blockIdx.x * (256 * PPT) + threadIdx.x;
    float* dx = disp + slot * g.slot_part;
    float* dy = dx + N;
    float* dz = dy + N;
    float* vx = vel + slot * g.slot_part;
    float* vy = vx + N;
    float* vz = vy + N;
    const int ds = g.log2ng - g.log2np, l2p = g.log2np, mp = (1 << l2p) - 1;
    const float4* f = force4 + slot * g.slot_mesh;
    const long long M = 1ll << (3 * g.log2ng);
    float p[PPT][3], u[PPT][3], acc[PPT][3];
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
            const long long ip = (long long)i0 + 256 * k + STATE_PREFETCH;
            if (ip < N) {
                prefetch_l2(dx + ip);
                prefetch_l2(dy + ip);
                prefetch_l2(dz + ip);
                prefetch_l2(vx + ip);
                prefetch_l2(vy + ip);
                prefetch_l2(vz + ip);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int i = i0 + 256 * k;
        const bool ok = i < N;
        // the state is touched once per step: stream it past the caches the gathers use
        u[k][0] = ok ? __ldcs(vx + i) : 0.f;
        u[k][1] = ok ? __ldcs(vy + i) : 0.f;
        u[k][2] = ok ? __ldcs(vz + i) : 0.f;
        p[k][0] = (ok ? __ldcs(dx + i) : 0.f) + tin * u[k][0];      // drift_1: X_half
        p[k][1] = (ok ? __ldcs(dy + i) : 0.f) + tin * u[k][1];
        p[k][2] = (ok ? __ldcs(dz + i) : 0.f) + tin * u[k][2];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[k][c] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int i = i0 + 256 * k;
        if (i >= N) continue;
        const int ix = i & mp, iy = (i >> l2p) & mp, iz = i >> (2 * l2p);
        {
            const AxisTaps ax = axis_taps<ORDER>(ix, ds, p[k][0] * g.inv_h);
            const AxisTaps ay = axis_taps<ORDER>(iy, ds, p[k][1] * g.inv_h);
            const AxisTaps az = axis_taps<ORDER>(iz, ds, p[k][2] * g.inv_h);
            gather3v<ORDER>(f, g.log2ng, ax, ay, az, acc[k]);
        }
        if (IL) {
            // second grid shifted by half a cell; average the two interpolants
            float acc1[3] = {0.f, 0.f, 0.f};
            const AxisTaps ax = axis_taps<ORDER>(ix, ds, p[k][0] * g.inv_h + 0.5f);
            const AxisTaps ay = axis_taps<ORDER>(iy, ds, p[k][1] * g.inv_h + 0.5f);
            const AxisTaps az = axis_taps<ORDER>(iz, ds, p[k][2] * g.inv_h + 0.5f);
            gather3v<ORDER>(f + M, g.log2ng, ax, ay, az, acc1);
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[k][c] = 0.5f * (acc[k][c] + acc1[c]);
        }
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int i = i0 + 256 * k;
        if (i >= N) continue;
        float vn[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) vn[c] = cf.alpha * u[k][c] + cf.kick * acc[k][c];   // kick
        __stcs(vx + i, vn[0]);
        __stcs(vy + i, vn[1]);
        __stcs(vz + i, vn[2]);
        __stcs(dx + i, p[k][0] + tout * vn[0]);                                        // drift_2 (+ next drift_1)
        __stcs(dy + i, p[k][1] + tout * vn[1]);
        __stcs(dz + i, p[k][2] + tout * vn[2]);
    }
}

// Interpolation + kick + drift_2 along Lagrangian columns (CIC, mesh = lattice,
// no interlacing).  A CTA takes a 32 x 8 x 8 tile of lattice sites; thread t walks
// the column of 8 sites at (x, y) = (ix0 + t % 32, iy0 + t / 32) upwards in z.
// The ORDER planes of force taps (ORDER x ORDER float4 each) of the previous
// particle stay in registers: when the next particle lies in the same (x, y)
// cell column, z-shifted by 0..ORDER-1 cells, the planes it shares are reused and
// only the new ones are gathered (a lattice column that has not crossed cells
// gathers one plane per particle instead of ORDER).  The next particle's state
// is loaded while the current one gathers.
template <int ORDER>
__global__ void __launch_bounds__(256, 3) k_interp_col(PmGeom g, float* __restrict__ disp, float* __restrict__ vel,
                                                    const SlotCoef* __restrict__ coef, int cstride,
                                                    const float4* __restrict__ force4, int predrift_in,
                                                    const SlotCoef* __restrict__ coef_next) {
    using TG = TileGeom<1>;
    constexpr int PPT = TG::PPT;
    static_assert(TG::DZ == 1, "column walk needs consecutive planes");
    const int slot = blockIdx.y;
    const SlotCoef cf = coef[slot * cstride];
    if (!cf.active) return;
    const float tin = predrift_in ? 0.f : cf.tau1;
    const float tout = cf.tau2 + (coef_next ? coef_next[slot * cstride].tau1 : 0.f);
    const int l2 = g.log2np, msk = (1 << l2) - 1;
    const int N = 1 << (3 * l2), plane = 1 << (2 * l2);
    float* dx = disp + slot * g.slot_part;
    float* dy = dx + N;
    float* dz = dy + N;
    float* vx = vel + slot * g.slot_part;
    float* vy = vx + N;
    float* vz = vy + N;
    const float4* f = force4 + slot * g.slot_mesh;
    const TG T(blockIdx.x, l2);
    const int i0 = (T.iz * (1 << l2) + T.iy) * (1 << l2) + T.ix;
    // L2 prefetch of the state of the tile STATE_TILES ahead (one line per lattice row and array)
    constexpr int STATE_TILES = 32;
    if (blockIdx.x + STATE_TILES < gridDim.x && threadIdx.x < 64) {
        const TG Tn(blockIdx.x + STATE_TILES, l2);
        const int r = threadIdx.x;
        const int ip = ((Tn.iz0 + r / 8) * (1 << l2) + Tn.iy0 + r % 8) * (1 << l2) + Tn.ix0;
        prefetch_l2(dx + ip);
        prefetch_l2(dy + ip);
        prefetch_l2(dz + ip);
        prefetch_l2(vx + ip);
        prefetch_l2(vy + ip);
        prefetch_l2(vz + ip);
    }
    // and of the force rows that tile's undisplaced cells (+1 cell) cover: 10 x 10
    // rows of 6 128-byte lines (8 float4 cells each), so that the walk's first
    // touches of force lines hit L2
    if (blockIdx.x + STATE_TILES < gridDim.x) {
        const TG Tn(blockIdx.x + STATE_TILES, l2);
        for (int r = threadIdx.x; r < 10 * 10 * 6; r += 256) {
            const int zr = r / 60, yr = (r / 6) % 10, seg = r % 6;
            const int z = (Tn.iz0 - 1 + zr) & msk, y = (Tn.iy0 - 1 + yr) & msk;
            const int x = ((Tn.ix0 >> 3) - 1 + seg) & (msk >> 3);   // line index along the row
            prefetch_l2(f + ((z << (2 * l2)) + (y << l2) + (x << 3)));
        }
    }
    float4 P[ORDER][ORDER][ORDER];   // [z plane][y][x] taps of the previous particle
#pragma unroll
    for (int k = 0; k < ORDER; ++k)
#pragma unroll
        for (int b = 0; b < ORDER; ++b)
#pragma unroll
            for (int a = 0; a < ORDER; ++a) P[k][b][a] = make_float4(0.f, 0.f, 0.f, 0.f);
    int pcx = -(1 << 30), pcy = 0, pcz = 0;
    float nd[3], nv[3];
    nd[0] = __ldcs(dx + i0);
    nd[1] = __ldcs(dy + i0);
    nd[2] = __ldcs(dz + i0);
    nv[0] = __ldcs(vx + i0);
    nv[1] = __ldcs(vy + i0);
    nv[2] = __ldcs(vz + i0);
#pragma unroll
    for (int p = 0; p < PPT; ++p) {
        const int i = i0 + p * plane;
        float u[3], x[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            u[c] = nv[c];
            x[c] = nd[c] + tin * u[c];             // drift_1: X_half
        }
        if (p + 1 < PPT) {
            const int j = i + plane;
            nd[0] = __ldcs(dx + j);
            nd[1] = __ldcs(dy + j);
            nd[2] = __ldcs(dz + j);
            nv[0] = __ldcs(vx + j);
            nv[1] = __ldcs(vy + j);
            nv[2] = __ldcs(vz + j);
        }
        const AxisTaps ax = axis_taps<ORDER>(T.ix, 0, x[0] * g.inv_h);
        const AxisTaps ay = axis_taps<ORDER>(T.iy, 0, x[1] * g.inv_h);
        const AxisTaps az = axis_taps<ORDER>(T.iz + p, 0, x[2] * g.inv_h);
        // planes shared with the previous particle: shift = az.c - pcz in [0, ORDER)
        const int shift = (ax.c == pcx && ay.c == pcy) ? az.c - pcz : ORDER;
        const bool keep = shift >= 0 && shift < ORDER;
#pragma unroll
        for (int k = 0; k + 1 < ORDER; ++k) {
#pragma unroll
            for (int b = 0; b < ORDER; ++b)
#pragma unroll
                for (int a = 0; a < ORDER; ++a) {
                    float4 v = P[k][b][a];
                    if (shift == 1) v = P[k + 1][b][a];
                    if (ORDER == 3 && k == 0 && shift == 2) v = P[ORDER - 1][b][a];
                    P[k][b][a] = v;
                }
        }
        int xo[ORDER], yo[ORDER];
#pragma unroll
        for (int a = 0; a < ORDER; ++a) {
            xo[a] = (ax.c + a) & msk;
            yo[a] = ((ay.c + a) & msk) << l2;
        }
#pragma unroll
        for (int k = 0; k < ORDER; ++k) {
            if (!keep || k + shift >= ORDER) {
                const int zo = ((az.c + k) & msk) << (2 * l2);
#pragma unroll
                for (int b = 0; b < ORDER; ++b)
#pragma unroll
                    for (int a = 0; a < ORDER; ++a) P[k][b][a] = __ldg(f + (zo + yo[b] + xo[a]));
            }
        }
        pcx = ax.c;
        pcy = ay.c;
        pcz = az.c;
        float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < ORDER; ++k)
#pragma unroll
            for (int b = 0; b < ORDER; ++b) {
                const float wzy = az.w[k] * ay.w[b];
#pragma unroll
                for (int a = 0; a < ORDER; ++a) {
                    const float w = wzy * ax.w[a];
                    acc[0] += w * P[k][b][a].x;
                    acc[1] += w * P[k][b][a].y;
                    acc[2] += w * P[k][b][a].z;
                }
            }
        float vn[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) vn[c] = cf.alpha * u[c] + cf.kick * acc[c];   // kick
        __stcs(vx + i, vn[0]);
        __stcs(vy + i, vn[1]);
        __stcs(vz + i, vn[2]);
        __stcs(dx + i, x[0] + tout * vn[0]);                                        // drift_2 (+ next drift_1)
        __stcs(dy + i, x[1] + tout * vn[1]);
        __stcs(dz + i, x[2] + tout * vn[2]);
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

// ------------------------------------------------------------------ gradient stencil
// g = -D1 phi with the finite-difference gradients of Table 2 applied in real
// space: order 2: 1/2 [-1 0 1]; order 4: 1/12 [1 -8 0 8 -1]; order 6:
// 1/60 [-1 9 -45 0 45 -9 1] (times 1/H).  Their Fourier transforms are the
// gradient kernels used in k-space, so this equals applying them there, with
// one inverse FFT (of the potential) instead of three.
template <int GO>
__global__ void __launch_bounds__(256) k_grad_stencil(int log2n, float inv_h, const float* __restrict__ phi,
                                                      long long phi_stride, float4* __restrict__ out,
                                                      long long f_stride) {
    constexpr int R = GO / 2;
    const float c1 = GO == 2 ? 0.5f : (GO == 4 ? 8.f / 12.f : 45.f / 60.f);
    const float c2 = GO == 4 ? -1.f / 12.f : -9.f / 60.f;
    const float c3 = 1.f / 60.f;
    const int n = 1 << log2n, msk = n - 1;
    const long long M = 1ll << (3 * log2n);
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const float* f = phi + blockIdx.y * phi_stride;
    const int x = (int)(j & msk), y = (int)((j >> log2n) & msk), z = (int)(j >> (2 * log2n));
    auto at = [&](int xx, int yy, int zz) -> float {
        return __ldg(&f[((long long)(zz & msk) << (2 * log2n)) + ((long long)(yy & msk) << log2n) + (xx & msk)]);
    };
    float g[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int dx = c == 0, dy = c == 1, dz = c == 2;
        float d = c1 * (at(x + dx, y + dy, z + dz) - at(x - dx, y - dy, z - dz));
        if (R >= 2) d += c2 * (at(x + 2 * dx, y + 2 * dy, z + 2 * dz) - at(x - 2 * dx, y - 2 * dy, z - 2 * dz));
        if (R >= 3) d += c3 * (at(x + 3 * dx, y + 3 * dy, z + 3 * dz) - at(x - 3 * dx, y - 3 * dy, z - 3 * dz));
        g[c] = -d * inv_h;
    }
    out[blockIdx.y * f_stride + j] = make_float4(g[0], g[1], g[2], 0.f);
}

// Same gradient through shared-memory planes: a CTA owns a 32 x 16 column of
// cells over GS_ZC consecutive planes.  It marches up in z: the potential of its
// own cells at z - R .. z + R sits in a register queue (the z derivative), plane
// z with an R-cell x/y halo sits in shared memory (the x and y derivatives), and
// the next plane's values are loaded while the current one is differentiated.
// Every potential value is read from global memory about once per CTA (plus the
// halo and the 2R planes before the column), instead of 3 * GO times.
constexpr int GS_TX = 32, GS_TY = 16, GS_ZC = 32;
template <int GO>
__global__ void __launch_bounds__(256) k_grad_stencil_t(int log2n, float inv_h, const float* __restrict__ phi,
                                                        long long phi_stride, float4* __restrict__ out,
                                                        long long f_stride) {
    constexpr int R = GO / 2, SX = GS_TX + 2 * R, SY = GS_TY + 2 * R;
    constexpr int NH = 2 * R * (GS_TX + GS_TY), HPT = (NH + 255) / 256;   // halo cells per plane, per thread
    const float c1 = (GO == 2 ? 0.5f : (GO == 4 ? 8.f / 12.f : 45.f / 60.f)) * inv_h;
    const float c2 = (GO == 4 ? -1.f / 12.f : -9.f / 60.f) * inv_h;
    const float c3 = (1.f / 60.f) * inv_h;
    __shared__ float s[2][SY][SX];
    const int n = 1 << log2n, msk = n - 1, l2n = 2 * log2n;
    const int nzc = n / GS_ZC;
    const int slot = blockIdx.z / nzc, z0 = (blockIdx.z % nzc) * GS_ZC;
    const int x0 = blockIdx.x * GS_TX, y0 = blockIdx.y * GS_TY;
    const float* f = phi + slot * phi_stride;
    float4* o = out + slot * f_stride;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;          // cells (tx, ty) and (tx, ty + 8)
    const int row0 = (((y0 + ty) & msk) << log2n) + ((x0 + tx) & msk);
    const int row1 = (((y0 + ty + 8) & msk) << log2n) + ((x0 + tx) & msk);
    // halo cells of this thread: shared-memory slot and in-plane offset
    int hs[HPT], hg[HPT];
#pragma unroll
    for (int k = 0; k < HPT; ++k) {
        const int h = threadIdx.x + 256 * k;
        int sr = 0, sc = 0, gx = 0, gy = 0;
        if (h < 2 * R * GS_TY) {
            const int side = h / (R * GS_TY), rem = h % (R * GS_TY), r = rem / R, c = rem % R;
            sr = r + R;
            sc = side ? GS_TX + R + c : c;
            gx = x0 + (side ? GS_TX + c : c - R);
            gy = y0 + r;
        } else if (h < NH) {
            const int h2 = h - 2 * R * GS_TY;
            const int side = h2 / (R * GS_TX), rem = h2 % (R * GS_TX), r = rem / GS_TX, c = rem % GS_TX;
            sr = side ? GS_TY + R + r : r;
            sc = c + R;
            gx = x0 + c;
            gy = y0 + (side ? GS_TY + r : r - R);
        }
        hs[k] = h < NH ? sr * SX + sc : -1;
        hg[k] = ((gy & msk) << log2n) + (gx & msk);
    }
    auto plane = [&](int z) { return (long long)(z & msk) << l2n; };
    // register queues of the column values at z - R .. z + R, and the halo of plane z
    float q0[2 * R + 1], q1[2 * R + 1], hv[HPT];
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k) {
        const long long p = plane(z0 - R + k);
        q0[k] = __ldg(f + p + row0);
        q1[k] = __ldg(f + p + row1);
    }
#pragma unroll
    for (int k = 0; k < HPT; ++k) hv[k] = hs[k] >= 0 ? __ldg(f + plane(z0) + hg[k]) : 0.f;
    for (int zi = 0; zi < GS_ZC; ++zi) {
        const int z = z0 + zi, b = zi & 1;
        float* sb = &s[b][0][0];
        sb[(ty + R) * SX + tx + R] = q0[R];
        sb[(ty + 8 + R) * SX + tx + R] = q1[R];
#pragma unroll
        for (int k = 0; k < HPT; ++k)
            if (hs[k] >= 0) sb[hs[k]] = hv[k];
        // next plane's loads in flight during this plane's differences
        float n0 = 0.f, n1 = 0.f;
        if (zi + 1 < GS_ZC) {
            const long long pn = plane(z + R + 1);
            n0 = __ldg(f + pn + row0);
            n1 = __ldg(f + pn + row1);
#pragma unroll
            for (int k = 0; k < HPT; ++k) hv[k] = hs[k] >= 0 ? __ldg(f + plane(z + 1) + hg[k]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const float* q = half ? q1 : q0;
            const int sy = ty + 8 * half + R, sx = tx + R;
            const float* srow = sb + sy * SX + sx;
            float gx = c1 * (srow[1] - srow[-1]);
            float gy = c1 * (srow[SX] - srow[-SX]);
            float gz = c1 * (q[R + 1] - q[R - 1]);
            if (R >= 2) {
                gx += c2 * (srow[2] - srow[-2]);
                gy += c2 * (srow[2 * SX] - srow[-2 * SX]);
                gz += c2 * (q[R + 2] - q[R - 2]);
            }
            if (R >= 3) {
                gx += c3 * (srow[3] - srow[-3]);
                gy += c3 * (srow[3 * SX] - srow[-3 * SX]);
                gz += c3 * (q[R + 3] - q[R - 3]);
            }
            o[plane(z) + (half ? row1 : row0)] = make_float4(-gx, -gy, -gz, 0.f);
        }
#pragma unroll
        for (int k = 0; k < 2 * R; ++k) {
            q0[k] = q0[k + 1];
            q1[k] = q1[k + 1];
        }
        q0[2 * R] = n0;
        q1[2 * R] = n1;
    }
}

// div[q][j] = sum_c D1_c s_c at every cell for three planar meshes s_c (q < nmesh,
// s slot stride s_stride floats, c-th mesh at c * M; div slot stride d_stride).
// Its transpose pairs with k_grad_stencil: D1 is antisymmetric, so the adjoint
// of g_c = -D1_c Lap^-1 rho is rho* = Lap^-1 sum_c D1_c g*_c.
template <int GO>
__global__ void __launch_bounds__(256) k_div_stencil(int log2n, float inv_h, const float* __restrict__ s3,
                                                     long long s_stride, float* __restrict__ div,
                                                     long long d_stride) {
    constexpr int R = GO / 2;
    const float c1 = GO == 2 ? 0.5f : (GO == 4 ? 8.f / 12.f : 45.f / 60.f);
    const float c2 = GO == 4 ? -1.f / 12.f : -9.f / 60.f;
    const float c3 = 1.f / 60.f;
    const int n = 1 << log2n, msk = n - 1;
    const long long M = 1ll << (3 * log2n);
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    const int x = (int)(j & msk), y = (int)((j >> log2n) & msk), z = (int)(j >> (2 * log2n));
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float* f = s3 + blockIdx.y * s_stride + c * M;
        auto at = [&](int xx, int yy, int zz) -> float {
            return __ldg(&f[((long long)(zz & msk) << (2 * log2n)) + ((long long)(yy & msk) << log2n) + (xx & msk)]);
        };
        const int dx = c == 0, dy = c == 1, dz = c == 2;
        float d = c1 * (at(x + dx, y + dy, z + dz) - at(x - dx, y - dy, z - dz));
        if (R >= 2) d += c2 * (at(x + 2 * dx, y + 2 * dy, z + 2 * dz) - at(x - 2 * dx, y - 2 * dy, z - 2 * dz));
        if (R >= 3) d += c3 * (at(x + 3 * dx, y + 3 * dy, z + 3 * dz) - at(x - 3 * dx, y - 3 * dy, z - 3 * dz));
        acc += d * inv_h;
    }
    div[blockIdx.y * d_stride + j] = acc;
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
                                                    const float4* __restrict__ force4, float* __restrict__ s3) {
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
    const float4* f = force4 + slot * M;
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
                const float4 gv = __ldg(&f[j]);
                const float g0 = gv.x, g1 = gv.y, g2 = gv.z;
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

// ------------------------------------------------------------------ forward mode
// Tangents of the DKD step (the JVP counterpart of App. C): the deposit
// pushes forward as rho'_j = sum_i sum_d X'_di dW(r_j - X_i)/dX_di, the force
// operator is linear (g' = G rho'), and the gather as
// A'_c = gather(g'_c) + sum_d X'_d d/dX_d gather(g_c).

// DRIFT = 1: X_half = X + tau1 V, X'_half = X' + tau1 V' (written back); then the
// deposit of X_half into rho and of its tangent into trho.  DRIFT = 0: no drift
// and nothing written back (P(k) tangents).
template <int ORDER, int DRIFT>
__global__ void __launch_bounds__(256) k_jvp_drift_deposit(PmGeom g, float* __restrict__ disp,
                                                           const float* __restrict__ vel, float* __restrict__ tdisp,
                                                           const float* __restrict__ tvel,
                                                           const SlotCoef* __restrict__ coef, int cstride,
                                                           float* __restrict__ rho, float* __restrict__ trho) {
    const int slot = blockIdx.y;
    const SlotCoef cf = coef[slot * cstride];
    if (!cf.active) return;
    const long long N = 1ll << (3 * g.log2np);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Lattice L = lattice_index(i, g.log2np);
    const long long o = slot * g.slot_part;
    float p[3], t[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        p[c] = disp[o + c * N + i];
        t[c] = tdisp[o + c * N + i];
        if (DRIFT) {
            p[c] += cf.tau1 * vel[o + c * N + i];
            t[c] += cf.tau1 * tvel[o + c * N + i];
            disp[o + c * N + i] = p[c];
            tdisp[o + c * N + i] = t[c];
        }
        t[c] *= g.inv_h;                            // d/dX = inv_h d/du
    }
    const int ds = g.log2ng - g.log2np;
    const AxisTaps ax = axis_taps<ORDER>(L.ix, ds, p[0] * g.inv_h);
    const AxisTaps ay = axis_taps<ORDER>(L.iy, ds, p[1] * g.inv_h);
    const AxisTaps az = axis_taps<ORDER>(L.iz, ds, p[2] * g.inv_h);
    const int ng = 1 << g.log2ng, msk = ng - 1;
    float* m = rho ? rho + slot * g.slot_mesh : nullptr;
    float* tm = trho + slot * g.slot_mesh;
#pragma unroll
    for (int c = 0; c < ORDER; ++c) {
        const long long zo = (long long)((az.c + c) & msk) * ng;
#pragma unroll
        for (int b = 0; b < ORDER; ++b) {
            const long long yo = (zo + ((ay.c + b) & msk)) * ng;
#pragma unroll
            for (int a = 0; a < ORDER; ++a) {
                const long long j = yo + ((ax.c + a) & msk);
                if (m) atomicAdd(&m[j], az.w[c] * ay.w[b] * ax.w[a]);
                const float dv = t[0] * ax.dw[a] * ay.w[b] * az.w[c] + t[1] * ax.w[a] * ay.dw[b] * az.w[c] +
                                 t[2] * ax.w[a] * ay.w[b] * az.dw[c];
                atomicAdd(&tm[j], dv);
            }
        }
    }
}

// At X_half: A = gather(g), A' = gather(g') + X'_half . grad gather(g); then the
// kick and drift_2 of the state and of its tangent.
template <int ORDER>
__global__ void __launch_bounds__(256) k_jvp_interp_kick(PmGeom g, float* __restrict__ disp, float* __restrict__ vel,
                                                         float* __restrict__ tdisp, float* __restrict__ tvel,
                                                         const SlotCoef* __restrict__ coef, int cstride,
                                                         const float4* __restrict__ force4,
                                                         const float4* __restrict__ tforce4) {
    const int slot = blockIdx.y;
    const SlotCoef cf = coef[slot * cstride];
    if (!cf.active) return;
    const long long N = 1ll << (3 * g.log2np);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const Lattice L = lattice_index(i, g.log2np);
    const long long o = slot * g.slot_part;
    float p[3], t[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        p[c] = disp[o + c * N + i];
        t[c] = tdisp[o + c * N + i];
    }
    const int ds = g.log2ng - g.log2np;
    const AxisTaps ax = axis_taps<ORDER>(L.ix, ds, p[0] * g.inv_h);
    const AxisTaps ay = axis_taps<ORDER>(L.iy, ds, p[1] * g.inv_h);
    const AxisTaps az = axis_taps<ORDER>(L.iz, ds, p[2] * g.inv_h);
    const int ng = 1 << g.log2ng, msk = ng - 1;
    const long long M = 1ll << (3 * g.log2ng);
    const float4* f = force4 + slot * M;
    const float4* tf = tforce4 + slot * M;
    float A[3] = {0.f, 0.f, 0.f}, At[3] = {0.f, 0.f, 0.f};
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
                // X'_half . grad of the tap weight (per unit length)
                const float dw = g.inv_h * (t[0] * ax.dw[a] * ay.w[b] * az.w[c] + t[1] * ax.w[a] * ay.dw[b] * az.w[c] +
                                            t[2] * ax.w[a] * ay.w[b] * az.dw[c]);
                const float4 gv = __ldg(&f[j]);
                const float4 tv = __ldg(&tf[j]);
                A[0] += w * gv.x;
                A[1] += w * gv.y;
                A[2] += w * gv.z;
                At[0] += w * tv.x + dw * gv.x;
                At[1] += w * tv.y + dw * gv.y;
                At[2] += w * tv.z + dw * gv.z;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float v = cf.alpha * vel[o + c * N + i] + cf.kick * A[c];
        const float vt = cf.alpha * tvel[o + c * N + i] + cf.kick * At[c];
        vel[o + c * N + i] = v;
        tvel[o + c * N + i] = vt;
        disp[o + c * N + i] = p[c] + cf.tau2 * v;
        tdisp[o + c * N + i] = t[c] + cf.tau2 * vt;
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

// 2LPT source from three real fields per slot (see pm_lpt2_source)
__global__ void k_lpt2_source(int pass, const float* __restrict__ t, float* __restrict__ mu, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* ts = t + blockIdx.y * 3 * n;
    float* m = mu + blockIdx.y * n;
    const float a = ts[i], b = ts[n + i], c = ts[2 * n + i];
    if (pass == 0) m[i] = a * b + a * c + b * c;
    else m[i] = (-3.f / 7.f) * (m[i] - (a * a + b * b + c * c));
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
    const int R = 1 << (g.log2ng - g.log2np > 0 ? g.log2ng - g.log2np : 0);
    const bool tiled = (g.log2ng - g.log2np == 0 && g.log2np >= 5) || (g.log2ng - g.log2np == 1 && g.log2np >= 4);
    if (tiled && order >= 2 && order <= 5) {
        const int np = 1 << g.log2np;
        const unsigned ntiles = (unsigned)((long long)(np / (32 / R)) * (np / (8 / R)) * (np / (8 / R)));
#define PM_DT(O, RR)                                                                                        \
    {                                                                                                       \
        const int smem = DepWindow<O>::CELLS * (int)sizeof(unsigned);                                          \
        static int resident[64];                                                                            \
        int dev = 0;                                                                                        \
        cudaGetDevice(&dev);                                                                                \
        if (dev < 0 || dev >= 64) dev = 0;                                                                  \
        if (!resident[dev]) {                                                                               \
            cudaFuncSetAttribute(k_deposit_tiled<O, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
            int per_sm = 0, sms = 0;                                                                        \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deposit_tiled<O, RR>, 256, smem);      \
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);                              \
            resident[dev] = per_sm * sms > 0 ? per_sm * sms : 1;                                            \
        }                                                                                                   \
        dim3 grid(ntiles < (unsigned)resident[dev] ? ntiles : (unsigned)resident[dev], nslots);             \
        k_deposit_tiled<O, RR><<<grid, 256, smem, st>>>(g, disp, vel, coef, coef_stride, shift_cells, rho,  \
                                                        (int)ntiles);                                            \
    }
        if (order == 2 && R == 1) PM_DT(2, 1)
        else if (order == 2) PM_DT(2, 2)
        else if (order == 3 && R == 1) PM_DT(3, 1)
        else if (order == 3) PM_DT(3, 2)
        else if (order == 4 && R == 1) PM_DT(4, 1)
        else if (order == 4) PM_DT(4, 2)
        else if (R == 1) PM_DT(5, 1)
        else PM_DT(5, 2)
#undef PM_DT
        return 0;
    }
    dim3 grid((unsigned)((N + 255) / 256), nslots);
    if (order == 2)
        k_deposit<2><<<grid, 256, 0, st>>>(g, disp, vel, coef, coef_stride, shift_cells, rho);
    else if (order == 3)
        k_deposit<3><<<grid, 256, 0, st>>>(g, disp, vel, coef, coef_stride, shift_cells, rho);
    else if (order == 4)
        k_deposit<4><<<grid, 256, 0, st>>>(g, disp, vel, coef, coef_stride, shift_cells, rho);
    else if (order == 5)
        k_deposit<5><<<grid, 256, 0, st>>>(g, disp, vel, coef, coef_stride, shift_cells, rho);
    else
        return -1;
    return 0;
}

int pm_interp_kick(int order, int interlace, const PmGeom& g, float* disp, float* vel, const SlotCoef* coef,
                   int coef_stride, const float4* force4, int nslots, cudaStream_t st, int predrift_in,
                   const SlotCoef* coef_next) {
    const long long N = 1ll << (3 * g.log2np);
    if (order == 2 && !interlace && g.log2ng == g.log2np && g.log2np >= 5) {
        dim3 gt((unsigned)(N / 2048), nslots);
        k_interp_col<2><<<gt, 256, 0, st>>>(g, disp, vel, coef, coef_stride, force4, predrift_in, coef_next);
        return 0;
    }
    const int ppt = ik_ppt(order);
    dim3 grid((unsigned)((N + 256 * ppt - 1) / (256 * ppt)), nslots);
#define PM_IK(O, I) k_interp_kick<O, I><<<grid, 256, 0, st>>>(g, disp, vel, coef, coef_stride, force4, predrift_in, coef_next)
    if (order == 2 && !interlace) PM_IK(2, 0);
    else if (order == 2 && interlace) PM_IK(2, 1);
    else if (order == 3 && !interlace) PM_IK(3, 0);
    else if (order == 3 && interlace) PM_IK(3, 1);
    else if (order == 4 && !interlace) PM_IK(4, 0);
    else if (order == 4 && interlace) PM_IK(4, 1);
    else if (order == 5 && !interlace) PM_IK(5, 0);
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
    else if (order == 4 && !interlace) PM_I(4, 0);
    else if (order == 4 && interlace) PM_I(4, 1);
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
    else if (order == 4) k_adj_drift_deposit<4><<<grid, 256, 0, st>>>(g, disp, vel, adisp, avel, coef, cstride, rho);
    else return -1;
    return 0;
}

int pm_adj_interp(int order, const PmGeom& g, const float* disp, float* vel, float* adisp, const float* avel,
                  const SlotCoef* coef, int cstride, const float4* force, float* s3, int nslots, cudaStream_t st) {
    const long long N = 1ll << (3 * g.log2np);
    dim3 grid((unsigned)((N + 255) / 256), nslots);
    if (order == 2) k_adj_interp<2><<<grid, 256, 0, st>>>(g, disp, vel, adisp, avel, coef, cstride, force, s3);
    else if (order == 3) k_adj_interp<3><<<grid, 256, 0, st>>>(g, disp, vel, adisp, avel, coef, cstride, force, s3);
    else if (order == 4) k_adj_interp<4><<<grid, 256, 0, st>>>(g, disp, vel, adisp, avel, coef, cstride, force, s3);
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
    else if (order == 4 && finish) PM_AG(4, 1);
    else if (order == 4) PM_AG(4, 0);
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

int pm_grad_stencil(int grad_order, int log2n, float inv_h, const float* phi, long long phi_stride, float4* force4,
                    long long f_stride, int nmesh, cudaStream_t st) {
    const long long M = 1ll << (3 * log2n);
    if (log2n >= 5) {
        const int n = 1 << log2n;
        dim3 gt(n / GS_TX, n / GS_TY, (n / GS_ZC) * nmesh);
        if (grad_order == 2) k_grad_stencil_t<2><<<gt, 256, 0, st>>>(log2n, inv_h, phi, phi_stride, force4, f_stride);
        else if (grad_order == 4) k_grad_stencil_t<4><<<gt, 256, 0, st>>>(log2n, inv_h, phi, phi_stride, force4, f_stride);
        else if (grad_order == 6) k_grad_stencil_t<6><<<gt, 256, 0, st>>>(log2n, inv_h, phi, phi_stride, force4, f_stride);
        else return -1;
        return 0;
    }
    dim3 grid((unsigned)((M + 255) / 256), nmesh);
    if (grad_order == 2) k_grad_stencil<2><<<grid, 256, 0, st>>>(log2n, inv_h, phi, phi_stride, force4, f_stride);
    else if (grad_order == 4) k_grad_stencil<4><<<grid, 256, 0, st>>>(log2n, inv_h, phi, phi_stride, force4, f_stride);
    else if (grad_order == 6) k_grad_stencil<6><<<grid, 256, 0, st>>>(log2n, inv_h, phi, phi_stride, force4, f_stride);
    else return -1;
    return 0;
}

int pm_div_stencil(int grad_order, int log2n, float inv_h, const float* s3, long long s_stride, float* div,
                   long long d_stride, int nmesh, cudaStream_t st) {
    const long long M = 1ll << (3 * log2n);
    dim3 grid((unsigned)((M + 255) / 256), nmesh);
    if (grad_order == 2) k_div_stencil<2><<<grid, 256, 0, st>>>(log2n, inv_h, s3, s_stride, div, d_stride);
    else if (grad_order == 4) k_div_stencil<4><<<grid, 256, 0, st>>>(log2n, inv_h, s3, s_stride, div, d_stride);
    else if (grad_order == 6) k_div_stencil<6><<<grid, 256, 0, st>>>(log2n, inv_h, s3, s_stride, div, d_stride);
    else return -1;
    return 0;
}

int pm_lpt2_source(int pass, const float* t, float* mu, long long n, int nslots, cudaStream_t st) {
    dim3 grid((unsigned)((n + 255) / 256), nslots);
    k_lpt2_source<<<grid, 256, 0, st>>>(pass, t, mu, n);
    return 0;
}

int pm_jvp_drift_deposit(int order, int drift, const PmGeom& g, float* disp, const float* vel, float* tdisp,
                         const float* tvel, const SlotCoef* coef, int cstride, float* rho, float* trho, int nslots,
                         cudaStream_t st) {
    const long long N = 1ll << (3 * g.log2np);
    dim3 grid((unsigned)((N + 255) / 256), nslots);
#define PM_JD(O, D) k_jvp_drift_deposit<O, D><<<grid, 256, 0, st>>>(g, disp, vel, tdisp, tvel, coef, cstride, rho, trho)
    if (order == 2) { if (drift) PM_JD(2, 1); else PM_JD(2, 0); }
    else if (order == 3) { if (drift) PM_JD(3, 1); else PM_JD(3, 0); }
    else if (order == 4) { if (drift) PM_JD(4, 1); else PM_JD(4, 0); }
    else return -1;
#undef PM_JD
    return 0;
}

int pm_jvp_interp_kick(int order, const PmGeom& g, float* disp, float* vel, float* tdisp, float* tvel,
                       const SlotCoef* coef, int cstride, const float4* force4, const float4* tforce4, int nslots,
                       cudaStream_t st) {
    const long long N = 1ll << (3 * g.log2np);
    dim3 grid((unsigned)((N + 255) / 256), nslots);
    if (order == 2) k_jvp_interp_kick<2><<<grid, 256, 0, st>>>(g, disp, vel, tdisp, tvel, coef, cstride, force4, tforce4);
    else if (order == 3) k_jvp_interp_kick<3><<<grid, 256, 0, st>>>(g, disp, vel, tdisp, tvel, coef, cstride, force4, tforce4);
    else if (order == 4) k_jvp_interp_kick<4><<<grid, 256, 0, st>>>(g, disp, vel, tdisp, tvel, coef, cstride, force4, tforce4);
    else return -1;
    return 0;
}
