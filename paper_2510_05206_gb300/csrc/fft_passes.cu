// Spectral passes of the PM force evaluation (Sec. 2.5, "Computing the forces"):
//   x pass   real rows <-> half-spectrum rows (R2C / C2R via a half-length complex FFT)
//   y pass   complex columns along y, in place
//   z pass   complex columns along z, fused with the Fourier-space operator:
//            force  (Poisson Green's function x gradient kernel, Table 2), 1 -> 3 spectra
//            force with an interlaced grid (Sec. 2.8), 2 -> 6 spectra
//            IC     (Zel'dovich displacement from white noise), 1 -> 3 spectra
//            P(k)   (binned |delta_k|^2 with FP64 per-bin sums), 1 -> bins
//            adjoint of the force operator (multiplier conj(m_c), summed), 3 -> 1
//            2LPT (second derivatives of psi1 from w^; psi2 from its source), 1 -> 3
// Transforms are unnormalised; normalisations are folded into the multipliers.
#include "fft_core.cuh"
#include "pm_kernels.h"

namespace {

using namespace pmfft;

// ---------------------------------------------------------------- x pass, R2C
// z[m] = x[2m] + i x[2m+1], Z = FFT_{n/2}(z),
// X[k] = (Z[k] + conj Z[n/2-k]) / 2 - i/2 exp(-2 pi i k / n) (Z[k] - conj Z[n/2-k]),  k = 0..n/2.
template <int LOG2N>
__global__ void __launch_bounds__(256) k_fft_x_r2c(const float* __restrict__ in, long long in_stride,
                                                   float2* __restrict__ out, long long out_stride,
                                                   const float2* __restrict__ twg, int clear_in) {
    constexpr int n = 1 << LOG2N, N = n / 2, P = N + SPEC_PAD;
    constexpr int ROWS = (2048 / N) < n * n ? (2048 / N) : n * n;
    constexpr int LS = N + 1;
    extern __shared__ float2 sm[];
    float2* tile = sm;
    float2* tw = sm + ROWS * LS;
    const int q = blockIdx.y;
    const long long row0 = (long long)blockIdx.x * ROWS;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    const float4* src = reinterpret_cast<const float4*>(in + q * in_stride + row0 * n);
    for (int i = threadIdx.x; i < ROWS * N / 2; i += blockDim.x) {
        const int r = i / (N / 2), c = i % (N / 2);
        const float4 v = src[i];
        tile[r * LS + 2 * c] = make_float2(v.x, v.y);
        tile[r * LS + 2 * c + 1] = make_float2(v.z, v.w);
    }
    if (clear_in) {
        // a consumed density mesh is left zeroed for the next deposit (after all the
        // loads above are issued: stores in the load loop would serialise them)
        __syncthreads();
        float4* dstz = reinterpret_cast<float4*>(const_cast<float*>(in) + q * in_stride + row0 * n);
        for (int i = threadIdx.x; i < ROWS * N / 2; i += blockDim.x) dstz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    fft_lines<N, ROWS, LS, 1, -1>(tile, tw, 2);
    float2* dst = out + q * out_stride + row0 * P;
    for (int i = threadIdx.x; i < ROWS * (N + 1); i += blockDim.x) {
        const int r = i / (N + 1), k = i % (N + 1);
        const float2 zk = tile[r * LS + (k == N ? 0 : k)];
        const float2 zc = cconj(tile[r * LS + (k == 0 ? 0 : N - k)]);
        const float2 e = cscale(cadd(zk, zc), 0.5f);
        const float2 o = cmul_i(cscale(csub(zk, zc), 0.5f), -1);   // (Z - conj)/(2i)
        dst[r * P + k] = cadd(e, cmul(tw[k], o));
    }
}

// ---------------------------------------------------------------- x pass, C2R
// Z[k] = X[k] + conj X[n/2-k] + i (X[k] - conj X[n/2-k]) exp(+2 pi i k / n), k < n/2;
// z = IFFT_{n/2}(Z) (unnormalised) gives x[2m] = Re z[m], x[2m+1] = Im z[m].
// EPI 0: out = x.  EPI 1: out = x, out2 = scale2 * x (Zel'dovich: V = psi1, Psi = D psi1).
template <int LOG2N, int EPI>
__global__ void __launch_bounds__(256) k_fft_x_c2r(const float2* __restrict__ in, long long in_stride,
                                                   float* __restrict__ out, long long out_stride,
                                                   float* __restrict__ out2, long long out2_stride,
                                                   float scale2, const float2* __restrict__ twg) {
    constexpr int n = 1 << LOG2N, N = n / 2, P = N + SPEC_PAD;
    constexpr int ROWS = (2048 / N) < n * n ? (2048 / N) : n * n;
    constexpr int LS = N + 1;
    extern __shared__ float2 sm[];
    float2* tile = sm;
    float2* tw = sm + ROWS * LS;
    const int q = blockIdx.y;
    const long long row0 = (long long)blockIdx.x * ROWS;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    const float2* src = in + q * in_stride + row0 * P;
    for (int i = threadIdx.x; i < ROWS * (N + 1); i += blockDim.x) {
        const int r = i / (N + 1), k = i % (N + 1);
        tile[r * LS + k] = src[r * P + k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ROWS * (N / 2 + 1); i += blockDim.x) {
        const int r = i / (N / 2 + 1), k = i % (N / 2 + 1);
        float2* t = tile + r * LS;
        const float2 a = t[k], b = t[N - k];
        // Z[k]
        const float2 ek = cadd(a, cconj(b));
        const float2 ok = cmul(csub(a, cconj(b)), cconj(tw[k]));
        const float2 zk = cadd(ek, cmul_i(ok, 1));
        if (k > 0 && k < N / 2) {
            const float2 em = cadd(b, cconj(a));
            const float2 om = cmul(csub(b, cconj(a)), cconj(tw[N - k]));
            t[N - k] = cadd(em, cmul_i(om, 1));
        }
        t[k] = zk;
    }
    __syncthreads();
    fft_lines<N, ROWS, LS, 1, 1>(tile, tw, 2);
    float4* dst = reinterpret_cast<float4*>(out + q * out_stride + row0 * n);
    float4* dst2 = EPI == 1 ? reinterpret_cast<float4*>(out2 + q * out2_stride + row0 * n) : nullptr;
    for (int i = threadIdx.x; i < ROWS * N / 2; i += blockDim.x) {
        const int r = i / (N / 2), c = i % (N / 2);
        const float2 z0 = tile[r * LS + 2 * c], z1 = tile[r * LS + 2 * c + 1];
        const float4 v = make_float4(z0.x, z0.y, z1.x, z1.y);
        dst[i] = v;
        if (EPI == 1) dst2[i] = make_float4(scale2 * v.x, scale2 * v.y, scale2 * v.z, scale2 * v.w);
    }
}


// ---------------------------------------------------------------- x pass, C2R x3 -> float4
// The three force spectra of one slot and grid, inverse transformed together and
// written interleaved as one float4 mesh (gx, gy, gz, 0): the interpolation then
// gathers one 16-byte value per tap.
template <int LOG2N>
__global__ void __launch_bounds__(768) k_fft_x_c2r3(const float2* __restrict__ in, long long comp_stride,
                                                    long long slot_stride, float4* __restrict__ out,
                                                    long long out_stride, const float2* __restrict__ twg) {
    constexpr int n = 1 << LOG2N, N = n / 2, P = N + SPEC_PAD;
    constexpr int ROWS = (2048 / N) < n * n ? (2048 / N) : n * n;
    constexpr int LS = N + 1;
    constexpr int L = 3 * ROWS;                         // lines: component-major, then row
    extern __shared__ float2 sm[];
    float2* tile = sm;
    float2* tw = sm + L * LS;
    const int q = blockIdx.y;
    const long long row0 = (long long)blockIdx.x * ROWS;
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    for (int i = threadIdx.x; i < L * (N + 1); i += blockDim.x) {
        const int line = i / (N + 1), k = i % (N + 1);
        const int c = line / ROWS, r = line % ROWS;
        tile[line * LS + k] = in[q * slot_stride + c * comp_stride + (row0 + r) * P + k];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < L * (N / 2 + 1); i += blockDim.x) {
        const int line = i / (N / 2 + 1), k = i % (N / 2 + 1);
        float2* t = tile + line * LS;
        const float2 a = t[k], b = t[N - k];
        const float2 ek = cadd(a, cconj(b));
        const float2 ok = cmul(csub(a, cconj(b)), cconj(tw[k]));
        const float2 zk = cadd(ek, cmul_i(ok, 1));
        if (k > 0 && k < N / 2) {
            const float2 em = cadd(b, cconj(a));
            const float2 om = cmul(csub(b, cconj(a)), cconj(tw[N - k]));
            t[N - k] = cadd(em, cmul_i(om, 1));
        }
        t[k] = zk;
    }
    __syncthreads();
    fft_lines<N, L, LS, 1, 1>(tile, tw, 2);
    float4* dst = out + q * out_stride + row0 * n;
    for (int i = threadIdx.x; i < ROWS * n; i += blockDim.x) {
        const int r = i / n, x = i % n;
        const int m = x >> 1;
        const float2 z0 = tile[(0 * ROWS + r) * LS + m];
        const float2 z1 = tile[(1 * ROWS + r) * LS + m];
        const float2 z2 = tile[(2 * ROWS + r) * LS + m];
        dst[i] = (x & 1) ? make_float4(z0.y, z1.y, z2.y, 0.f) : make_float4(z0.x, z1.x, z2.x, 0.f);
    }
}

// ---------------------------------------------------------------- column tiles
// A column tile is COL_TILE adjacent kx columns of one z plane (y pass) or one
// y row (z pass), all n elements along the transform axis.  The first FFT stage
// reads it straight from global memory and the last stage writes it straight
// back (fft_io), so a tile makes two shared-memory round trips per element for
// n = 512 instead of four.
// y rows per CTA of the P(k) z pass (amortises its accumulator clear / reduce / flush;
// the forward-mode pass, with two transforms per row, keeps one row to stay in registers)
__host__ __device__ constexpr int z_pk_rows(int log2n, bool two) {
    return two ? 1 : (log2n >= 9 ? 8 : (log2n == 8 ? 2 : 1));
}
__host__ __device__ constexpr int col_min_blocks(int log2n) { return (1024 >> log2n) > 32 ? 32 : ((1024 >> log2n) < 1 ? 1 : (1024 >> log2n)); }

// y pass: grid (tile groups, n planes, meshes).  A CTA transforms Y_TPC column
// tiles of one plane in turn, with the next tile's first-stage loads in flight
// during the current tile's transform.
constexpr int Y_TPC = 3;
template <int LOG2N, int DIR>
__global__ void __launch_bounds__(1 << LOG2N, col_min_blocks(LOG2N)) k_fft_y(float2* __restrict__ data, long long stride,
                                                                            const float2* __restrict__ twg) {
    constexpr int n = 1 << LOG2N, P = n / 2 + SPEC_PAD, NT = P / COL_TILE;
    extern __shared__ float2 sm[];
    float2* tw = sm;
    const ColTile tile{sm + n};
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    float2* base = data + blockIdx.z * stride + (long long)blockIdx.y * n * P;
    const int t0 = blockIdx.x * Y_TPC, t1 = t0 + Y_TPC < NT ? t0 + Y_TPC : NT;
    float2 nxt[8];
    fft_first_load<n, COL_TILE>(GCols{base + t0 * COL_TILE, P}, nxt);
    for (int t = t0; t < t1; ++t) {
        float2 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = nxt[k];
        if (t + 1 < t1) fft_first_load<n, COL_TILE>(GCols{base + (t + 1) * COL_TILE, P}, nxt);
        // the first stage needs no twiddles; the barrier after it publishes them
        const GCols g{base + t * COL_TILE, P};
        fft_pre<n, COL_TILE, DIR, false>(v, g, tile, tw, 1);
        __syncthreads();   // the next tile's first stage overwrites what the last stage read
    }
}

// ---------------------------------------------------------------- z pass
struct ZArgs {
    const float2* in[3];      // input spectra (slot 0); slot b adds b * slot_stride
    float2* out[6];           // output spectra
    long long slot_stride;    // complex elements between slots of one spectrum buffer
    const float2* tw;         // exp(-2 pi i m / n), m < n
    const float* lap1;        // 1D Laplacian kernel per bin (Table 2)
    const float* grad1;       // Im of the 1D gradient kernel per bin, 0 on the Nyquist bin
    const float* dec1;        // deconvolution 1 / W^(k)^2 per bin of one axis, or NULL
    const float* ictab;       // IC: sqrt(P(k) M / L^3) / (D(1) k^2) / M per integer k^2 index (0 if masked)
    double* pk_out;           // P(k): [slot][3][nbins] (sum w|d|^2, sum w|k|, sum w)
    int nbins;
    float scale;              // overall factor of the multiplier
    float kf;                 // 2 pi / L
};

enum { Z_FORCE = 0, Z_FORCE_IL = 1, Z_IC = 2, Z_PK = 3, Z_ADJ = 4, Z_IC_ADJ = 5, Z_POT = 6, Z_POT_IL = 7,
       Z_IC_D2 = 8, Z_IC_O2 = 9, Z_LPT2 = 10, Z_PKX = 11, Z_DEC = 16 };

// Last-stage store of the IC z pass: column l of the inverse transform G goes to
// the x and y displacement spectra as i kx G and i my G.
struct IcXYStore {
    float2* ox;
    float2* oy;
    long long es;
    int kx0;
    float my;
    __device__ __forceinline__ void operator()(int l, int e, float2 v) const {
        ox[e * es + l] = cmul_i(cscale(v, (float)(kx0 + l)), 1);
        oy[e * es + l] = cmul_i(cscale(v, my), 1);
    }
};

// MODE_DEC = mode | Z_DEC: the mode's multiplier also divides by the squared mass
// assignment kernel (deconvolution tables in a.dec1), compiled only where used.
template <int LOG2N, int MODE_DEC>
__global__ void __launch_bounds__(1 << LOG2N, col_min_blocks(LOG2N)) k_fft_z(ZArgs a) {
    constexpr int MODE = MODE_DEC & (Z_DEC - 1);
    constexpr bool deconv = (MODE_DEC & Z_DEC) != 0;
    constexpr int n = 1 << LOG2N, P = n / 2 + SPEC_PAD;
    constexpr int TE = col_tile_elems(n);
    constexpr long long ES = (long long)n * P;      // z stride (complex)
    extern __shared__ float2 sm[];
    float2* tw = sm;
    float* lap = reinterpret_cast<float*>(sm + n);
    float* grad = lap + n;
    float* dec = grad + n;                          // deconvolution: n floats = n/2 float2
    constexpr int T0 = 2 * n + (deconv ? n / 2 : 0);   // tiles after the tables
    const ColTile A{sm + T0};
    const ColTile B{sm + T0 + TE};
    const ColTile A2{sm + T0 + 2 * TE};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        tw[i] = a.tw[i];
        if (MODE == Z_FORCE || MODE == Z_FORCE_IL || MODE == Z_ADJ || MODE == Z_POT || MODE == Z_POT_IL) {
            lap[i] = a.lap1[i];
            grad[i] = a.grad1[i];
            if (deconv) dec[i] = a.dec1[i];
        }
    }
    if constexpr (MODE == Z_PK || MODE == Z_PKX) {
        // sum over the modes of each bin of w |delta^|^2 (w = 2 for 0 < kx < n/2, the
        // half spectrum standing for +-kx), FP64 per bin; Z_PKX (forward mode of P(k))
        // sums w 2 Re(conj(delta^) delta'^) with delta'^ the transform of in[1].
        // A CTA takes the same kx columns of ROWS consecutive y rows, so its
        // accumulators are cleared, reduced and flushed once for all of them: runs of
        // equal bin along kz are summed per thread in FP32, added to per-warp (or one
        // shared set of) FP64 accumulators in shared memory, and each CTA adds its
        // non-zero bins to the output with one global atomic each.  Mode counts and
        // mean |k| per bin depend on the mesh only and are tabulated on the host.
        double* acc = reinterpret_cast<double*>(B.s);
        constexpr int NW = (1 << LOG2N) >= 32 ? (1 << LOG2N) / 32 : 1;
        const bool priv = NW * a.nbins <= TE;
        const int nacc = priv ? NW * a.nbins : a.nbins;
        for (int i = threadIdx.x; i < nacc; i += blockDim.x) acc[i] = 0.0;
        __syncthreads();
        double* wacc = priv ? acc + (threadIdx.x >> 5) * a.nbins : acc;
        const int slot = blockIdx.z;
        const int kx0 = blockIdx.x * COL_TILE;
        // thread: column l, COL_TILE consecutive kz planes.  Along a column |k| is monotone
        // on each side of kz = n/2, so the bin changes rarely.
        constexpr int CH = COL_TILE;                       // n * COL_TILE elements / n threads
        const int l = threadIdx.x % COL_TILE, e0 = (threadIdx.x / COL_TILE) * CH;
        const int kx = kx0 + l;
        const float wx = (kx == 0 || kx == n / 2) ? 1.f : 2.f;
        constexpr int ROWS = z_pk_rows(LOG2N, MODE == Z_PKX);
#pragma unroll 1
        for (int yy = 0; yy < ROWS; ++yy) {
            const int y = blockIdx.y * ROWS + yy;
            const long long off = slot * a.slot_stride + (long long)y * P + kx0;
            const int my = freq_index(y, n);
            fft_io<n, COL_TILE, -1, false, true>(GCols{const_cast<float2*>(a.in[0]) + off, ES}, A, A, tw, 1);
            if (MODE == Z_PKX) {
                __syncthreads();
                fft_io<n, COL_TILE, -1, false, true>(GCols{const_cast<float2*>(a.in[1]) + off, ES}, A2, A2, tw, 1);
            }
            __syncthreads();
            if (kx <= n / 2) {
                const int kxy = kx * kx + my * my;
                int cur = -1;
                float run = 0.f;
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                    const int e = e0 + k, mz = freq_index(e, n);
                    // bin floor(|m| - 1/2) of the integer |m|^2 <= 3 (n/2)^2 < 2^24: the float
                    // square root is correctly rounded and |m| never lies within 1e-4 of a
                    // bin edge, so this equals the exact bin (0 for |m| = 0 gives -1)
                    int bk = (int)floorf(sqrtf((float)(kxy + mz * mz)) - 0.5f);
                    bk = bk < a.nbins ? bk : -1;
                    const float2 d = A(l, e);
                    const float2 dt = MODE == Z_PKX ? A2(l, e) : d;
                    if (bk != cur) {
                        if (cur >= 0) atomicAdd(&wacc[cur], (double)run);
                        cur = bk;
                        run = 0.f;
                    }
                    run += (MODE == Z_PKX ? 2.f * wx : wx) * (d.x * dt.x + d.y * dt.y);
                }
                if (cur >= 0) atomicAdd(&wacc[cur], (double)run);
            }
            __syncthreads();   // the next row's transform overwrites A
        }
        if (priv)
            for (int i = threadIdx.x; i < a.nbins; i += blockDim.x) {
                double sum = 0.0;
                for (int w = 0; w < NW; ++w) sum += acc[w * a.nbins + i];
                acc[i] = sum;   // each i is owned by one thread: reading row 0 before writing it is safe
            }
        __syncthreads();
        double* dst = a.pk_out + (long long)slot * a.nbins;
        for (int i = threadIdx.x; i < a.nbins; i += blockDim.x)
            if (acc[i] != 0.0) atomicAdd(&dst[i], acc[i]);
        return;
    }

    const int slot = blockIdx.z;
    const int y = blockIdx.y;
    const int kx0 = blockIdx.x * COL_TILE;
    const long long off = slot * a.slot_stride + (long long)y * P + kx0;
    const int my = freq_index(y, n);
    const GCols in0{const_cast<float2*>(a.in[0]) + off, ES};

    if (MODE == Z_ADJ || MODE == Z_IC_ADJ) {
        // Z_ADJ: sum_c conj(m_c) x_c^, m_c = -i D1(k_c) / K_lap(k) * scale => conj(m_c) = +i D1 / K * scale
        // Z_IC_ADJ: sum_c conj(i k_c T(k^2)) x_c^ = -i T sum_c k_c x_c^ (every Nyquist plane zero)
        fft_io<n, COL_TILE, -1, false, true>(in0, A, A, tw, 1);
        __syncthreads();
        fft_io<n, COL_TILE, -1, false, true>(GCols{const_cast<float2*>(a.in[1]) + off, ES}, B, B, tw, 1);
        __syncthreads();
        fft_io<n, COL_TILE, -1, false, true>(GCols{const_cast<float2*>(a.in[2]) + off, ES}, A2, A2, tw, 1);
        __syncthreads();
        auto comb = [&](int l, int e) -> float2 {
            const int kx = kx0 + l;
            float2 r = make_float2(0.f, 0.f);
            if (MODE == Z_ADJ && kx <= n / 2 && (kx | y | e)) {
                float inv = a.scale / (lap[kx] + lap[y] + lap[e]);
                if constexpr (deconv) inv *= dec[kx] * dec[y] * dec[e];
                const float2 s3 = cadd(cadd(cscale(A(l, e), grad[kx]), cscale(B(l, e), grad[y])), cscale(A2(l, e), grad[e]));
                r = cmul_i(cscale(s3, inv), 1);
            }
            if (MODE == Z_IC_ADJ && kx < n / 2 && y != n / 2 && e != n / 2) {
                const int mz = freq_index(e, n);
                const float f = a.kf * __ldg(&a.ictab[kx * kx + my * my + mz * mz]);
                const float2 s3 = cadd(cadd(cscale(A(l, e), (float)kx), cscale(B(l, e), (float)my)), cscale(A2(l, e), (float)mz));
                r = cmul_i(cscale(s3, f), -1);
            }
            return r;
        };
        fft_io<n, COL_TILE, 1, true, false>(comb, GCols{a.out[0] + off, ES}, A, tw, 1);
        return;
    }

    if constexpr (MODE == Z_POT) {
        // potential phi^ = scale * delta^ / K_lap(k): the forward transform's last stage
        // leaves each thread the elements the inverse's first stage takes, so the
        // multiplier is applied in registers between them (no shared-memory round trip)
        fft_head<n, COL_TILE, -1>(in0, A, tw, 1);
        float2 v[8];
        fft_tail_regs<n, COL_TILE, -1>(A, v, tw, 1);
        const int l = threadIdx.x % COL_TILE, j = threadIdx.x / COL_TILE;
        const int kx = kx0 + l;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int e = j + r * (n / 8);
            float f = 0.f;
            if (kx <= n / 2 && (kx | y | e) != 0) {
                f = a.scale / (lap[kx] + lap[y] + lap[e]);
                if constexpr (deconv) f *= dec[kx] * dec[y] * dec[e];
            }
            v[r] = cscale(v[r], f);
        }
        fft_pre<n, COL_TILE, 1, false>(v, GCols{a.out[0] + off, ES}, B, tw, 1);
        return;
    }

    if constexpr (MODE == Z_IC) {
        // the factor kf T(k^2) that the three components share is applied once, between
        // the forward transform's last stage (in registers) and its store to A; the
        // components then only multiply by i m_c
        fft_head<n, COL_TILE, -1>(in0, A, tw, 1);
        float2 v[8];
        fft_tail_regs<n, COL_TILE, -1>(A, v, tw, 1);
        const int l = threadIdx.x % COL_TILE, j = threadIdx.x / COL_TILE;
        const int kx = kx0 + l;
        __syncthreads();   // every thread has read its last-stage inputs from A
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int e = j + r * (n / 8), mz = freq_index(e, n);
            // zero on every Nyquist plane and in the padding columns
            const float f = (kx < n / 2 && y != n / 2 && e != n / 2)
                                ? a.kf * __ldg(&a.ictab[kx * kx + my * my + mz * mz]) : 0.f;
            A(l, e, cscale(v[r], f));
        }
    } else {
        fft_io<n, COL_TILE, -1, false, true>(in0, A, A, tw, 1);
    }
    if (MODE == Z_FORCE_IL || MODE == Z_POT_IL) {
        __syncthreads();
        fft_io<n, COL_TILE, -1, false, true>(GCols{const_cast<float2*>(a.in[1]) + off, ES}, A2, A2, tw, 1);
    }
    __syncthreads();

    if (MODE == Z_POT || MODE == Z_POT_IL) {
        // potential phi^ = scale * delta^ / K_lap(k) (k = 0 -> 0); the gradient of a
        // finite-difference order is applied afterwards as a real-space stencil.
        // Interlaced: delta^ = (d0^ + exp(i k.s) d1^)/2 and phi^ on both grids (phi^ and
        // phi^ exp(-i k.s)), every Nyquist plane zeroed.
        const int ngrid = MODE == Z_POT_IL ? 2 : 1;
        for (int gi = 0; gi < ngrid; ++gi) {
            auto mult = [&](int l, int e) -> float2 {
                const int kx = kx0 + l;
                float2 r = make_float2(0.f, 0.f);
                if (kx > n / 2 || (kx | y | e) == 0) return r;
                float2 d = A(l, e);
                if (MODE == Z_POT_IL) {
                    if (kx == n / 2 || y == n / 2 || e == n / 2) return r;
                    const int mz = freq_index(e, n);
                    float sn, cs;
                    sincospif((float)(kx + my + mz) / n, &sn, &cs);
                    d = cscale(cadd(d, cmul(make_float2(cs, sn), A2(l, e))), 0.5f);
                    if (gi == 1) d = cmul(d, make_float2(cs, -sn));
                }
                float f = a.scale / (lap[kx] + lap[y] + lap[e]);
                if constexpr (deconv) f *= dec[kx] * dec[y] * dec[e];
                return cscale(d, f);
            };
            fft_io<n, COL_TILE, 1, false, false>(mult, GCols{a.out[gi] + off, ES}, B, tw, 1);
            __syncthreads();
        }
        return;
    }

    if constexpr (MODE == Z_IC) {
        // psi1_c^ = i m_c (kf T w^) with A = kf T w^: along a z column m_x and m_y are
        // constants, so the x and y components are i kx and i my times ONE inverse
        // transform of A (two stores from its last stage); z needs its own
        const IcXYStore sxy{a.out[0] + off, a.out[1] + off, ES, kx0, (float)my};
        fft_io<n, COL_TILE, 1, false, false>(A, sxy, B, tw, 1);
        __syncthreads();
        auto mult_z = [&](int l, int e) -> float2 {
            return cmul_i(cscale(A(l, e), (float)freq_index(e, n)), 1);
        };
        fft_io<n, COL_TILE, 1, false, false>(mult_z, GCols{a.out[2] + off, ES}, B, tw, 1);
        return;
    }

    const int ncomp = MODE == Z_FORCE_IL ? 6 : 3;
    for (int c = 0; c < ncomp; ++c) {
        const int axis = c % 3;
        auto mult = [&](int l, int e) -> float2 {
            const int kx = kx0 + l;
            float2 r = make_float2(0.f, 0.f);
            if (kx > n / 2) return r;
            const int mz = freq_index(e, n);
            if (MODE == Z_IC_D2 || MODE == Z_IC_O2) {
                // second derivatives of psi1 for the 2LPT source (Eq. LPT_kernels):
                // psi1_i,j^ = i k_j psi1_i^ = -k_i k_j T(k^2) w^; D2: (xx, yy, zz), O2: (xy, xz, yz)
                if (kx != n / 2 && y != n / 2 && e != n / 2) {
                    const int m3[3] = {kx, my, mz};
                    const int i0 = MODE == Z_IC_D2 ? axis : (axis == 2 ? 1 : 0);
                    const int i1 = MODE == Z_IC_D2 ? axis : (axis == 0 ? 1 : 2);
                    const float f = -a.kf * a.kf * (float)(m3[i0] * m3[i1]) *
                                    __ldg(&a.ictab[kx * kx + my * my + mz * mz]);
                    r = cscale(A(l, e), f);
                }
                return r;
            }
            if (MODE == Z_LPT2) {
                // psi2_c^ = Lap^-1 grad_c L2^ = -i k_c L2^ / k^2 (scale = 1/M), zero at k = 0 and on
                // every Nyquist plane
                const int m2 = kx * kx + my * my + mz * mz;
                if (m2 != 0 && kx != n / 2 && y != n / 2 && e != n / 2) {
                    const int mc = axis == 0 ? kx : (axis == 1 ? my : mz);
                    const float f = a.scale * (float)mc / (a.kf * (float)m2);
                    r = cmul_i(cscale(A(l, e), f), -1);
                }
                return r;
            }
            // g_c^ = -i D1(k_c) / K_lap(k) * scale * delta^   (k = 0 -> 0)
            const int bc = axis == 0 ? kx : (axis == 1 ? y : e);
            float2 d = A(l, e);
            bool keep = (kx | y | e) != 0;
            if (MODE == Z_FORCE_IL) {
                // delta^ = (d0^ + exp(i k.s) d1^) / 2, s = H/2 (1,1,1); every Nyquist plane zeroed
                keep = keep && kx != n / 2 && y != n / 2 && e != n / 2;
                float sn, cs;
                sincospif((float)(kx + my + mz) / n, &sn, &cs);
                d = cscale(cadd(d, cmul(make_float2(cs, sn), A2(l, e))), 0.5f);
                if (c >= 3) d = cmul(d, make_float2(cs, -sn));   // grid 1: g^ exp(-i k.s)
            }
            if (keep) {
                float f = -grad[bc] * a.scale / (lap[kx] + lap[y] + lap[e]);
                if constexpr (deconv) f *= dec[kx] * dec[y] * dec[e];
                r = cmul_i(cscale(d, f), 1);
            }
            return r;
        };
        fft_io<n, COL_TILE, 1, false, false>(mult, GCols{a.out[c] + off, ES}, B, tw, 1);
        __syncthreads();
    }
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int LOG2N>
int rows_per_cta() {
    constexpr int n = 1 << LOG2N, N = n / 2;
    return (2048 / N) < n * n ? (2048 / N) : n * n;
}

template <int LOG2N>
void launch_x_r2c(const float* in, long long in_stride, float2* out, long long out_stride, int nmesh,
                  const float2* tw, int clear_in, cudaStream_t st) {
    constexpr int n = 1 << LOG2N, N = n / 2;
    const int rows = rows_per_cta<LOG2N>();
    const size_t smem = (size_t)(rows * (N + 1) + n) * sizeof(float2);
    set_smem(k_fft_x_r2c<LOG2N>, smem);
    dim3 grid(n * n / rows, nmesh);
    k_fft_x_r2c<LOG2N><<<grid, 256, smem, st>>>(in, in_stride, out, out_stride, tw, clear_in);
}

template <int LOG2N>
void launch_x_c2r(const float2* in, long long in_stride, float* out, long long out_stride, float* out2,
                  long long out2_stride, float scale2, int nmesh, const float2* tw, cudaStream_t st) {
    constexpr int n = 1 << LOG2N, N = n / 2;
    const int rows = rows_per_cta<LOG2N>();
    const size_t smem = (size_t)(rows * (N + 1) + n) * sizeof(float2);
    dim3 grid(n * n / rows, nmesh);
    if (out2) {
        set_smem(k_fft_x_c2r<LOG2N, 1>, smem);
        k_fft_x_c2r<LOG2N, 1><<<grid, 256, smem, st>>>(in, in_stride, out, out_stride, out2, out2_stride, scale2, tw);
    } else {
        set_smem(k_fft_x_c2r<LOG2N, 0>, smem);
        k_fft_x_c2r<LOG2N, 0><<<grid, 256, smem, st>>>(in, in_stride, out, out_stride, out2, out2_stride, scale2, tw);
    }
}

template <int LOG2N>
void launch_x_c2r3(const float2* in, long long comp_stride, long long slot_stride, float4* out, long long out_stride,
                   int nmesh, const float2* tw, cudaStream_t st) {
    constexpr int n = 1 << LOG2N, N = n / 2;
    const int rows = rows_per_cta<LOG2N>();
    const size_t smem = (size_t)(3 * rows * (N + 1) + n) * sizeof(float2);
    set_smem(k_fft_x_c2r3<LOG2N>, smem);
    dim3 grid(n * n / rows, nmesh);
    k_fft_x_c2r3<LOG2N><<<grid, 768, smem, st>>>(in, comp_stride, slot_stride, out, out_stride, tw);
}

template <int LOG2N>
void launch_y(float2* data, long long stride, int nmesh, int dir, const float2* tw, cudaStream_t st) {
    constexpr int n = 1 << LOG2N;
    const size_t smem = (size_t)(col_tile_elems(n) + n) * sizeof(float2);
    constexpr int NT = (n / 2 + SPEC_PAD) / COL_TILE;
    dim3 grid((NT + Y_TPC - 1) / Y_TPC, n, nmesh);
    if (dir < 0) {
        set_smem(k_fft_y<LOG2N, -1>, smem);
        k_fft_y<LOG2N, -1><<<grid, n, smem, st>>>(data, stride, tw);
    } else {
        set_smem(k_fft_y<LOG2N, 1>, smem);
        k_fft_y<LOG2N, 1><<<grid, n, smem, st>>>(data, stride, tw);
    }
}

template <int LOG2N, int MODE>
void launch_z_mode(const ZArgs& a, int nslots, cudaStream_t st) {
    constexpr int n = 1 << LOG2N;
    constexpr int M = MODE & (Z_DEC - 1);
    const int ntile = (M == Z_FORCE_IL || M == Z_ADJ || M == Z_IC_ADJ || M == Z_POT_IL || M == Z_PKX) ? 3 : 2;
    const size_t smem = (size_t)(ntile * col_tile_elems(n) + 2 * n + ((MODE & Z_DEC) ? n / 2 : 0)) * sizeof(float2);
    dim3 grid(n / 2 / COL_TILE + 1, (M == Z_PK || M == Z_PKX) ? n / z_pk_rows(LOG2N, M == Z_PKX) : n, nslots);
    set_smem(k_fft_z<LOG2N, MODE>, smem);
    k_fft_z<LOG2N, MODE><<<grid, n, smem, st>>>(a);
}

template <int LOG2N>
void launch_z(int mode, const ZArgs& a, int nslots, cudaStream_t st) {
    const bool dec = a.dec1 != nullptr;
    switch (mode) {
        case Z_FORCE:
            if (dec) launch_z_mode<LOG2N, Z_FORCE | Z_DEC>(a, nslots, st);
            else launch_z_mode<LOG2N, Z_FORCE>(a, nslots, st);
            break;
        case Z_FORCE_IL:
            if (dec) launch_z_mode<LOG2N, Z_FORCE_IL | Z_DEC>(a, nslots, st);
            else launch_z_mode<LOG2N, Z_FORCE_IL>(a, nslots, st);
            break;
        case Z_IC: launch_z_mode<LOG2N, Z_IC>(a, nslots, st); break;
        case Z_IC_D2: launch_z_mode<LOG2N, Z_IC_D2>(a, nslots, st); break;
        case Z_IC_O2: launch_z_mode<LOG2N, Z_IC_O2>(a, nslots, st); break;
        case Z_LPT2: launch_z_mode<LOG2N, Z_LPT2>(a, nslots, st); break;
        case Z_PK: launch_z_mode<LOG2N, Z_PK>(a, nslots, st); break;
        case Z_PKX: launch_z_mode<LOG2N, Z_PKX>(a, nslots, st); break;
        case Z_ADJ:
            if (dec) launch_z_mode<LOG2N, Z_ADJ | Z_DEC>(a, nslots, st);
            else launch_z_mode<LOG2N, Z_ADJ>(a, nslots, st);
            break;
        case Z_IC_ADJ: launch_z_mode<LOG2N, Z_IC_ADJ>(a, nslots, st); break;
        case Z_POT:
            if (dec) launch_z_mode<LOG2N, Z_POT | Z_DEC>(a, nslots, st);
            else launch_z_mode<LOG2N, Z_POT>(a, nslots, st);
            break;
        case Z_POT_IL:
            if (dec) launch_z_mode<LOG2N, Z_POT_IL | Z_DEC>(a, nslots, st);
            else launch_z_mode<LOG2N, Z_POT_IL>(a, nslots, st);
            break;
    }
}

}  // namespace

// ---------------------------------------------------------------- host dispatch
#define PM_DISPATCH_LOG2N(L2, CALL)                 \
    switch (L2) {                                   \
        case 4: { constexpr int LG = 4; CALL; } break;  \
        case 5: { constexpr int LG = 5; CALL; } break;  \
        case 6: { constexpr int LG = 6; CALL; } break;  \
        case 7: { constexpr int LG = 7; CALL; } break;  \
        case 8: { constexpr int LG = 8; CALL; } break;  \
        case 9: { constexpr int LG = 9; CALL; } break;  \
        case 10: { constexpr int LG = 10; CALL; } break; \
        default: return -1;                         \
    }

int pm_fft_r2c_x(int log2n, const float* in, long long in_stride, float2* out, long long out_stride, int nmesh,
                 const float2* tw, cudaStream_t st, int clear_in) {
    PM_DISPATCH_LOG2N(log2n, (launch_x_r2c<LG>(in, in_stride, out, out_stride, nmesh, tw, clear_in, st)));
    return 0;
}

int pm_fft_c2r_x(int log2n, const float2* in, long long in_stride, float* out, long long out_stride, float* out2,
                 long long out2_stride, float scale2, int nmesh, const float2* tw, cudaStream_t st) {
    PM_DISPATCH_LOG2N(log2n, (launch_x_c2r<LG>(in, in_stride, out, out_stride, out2, out2_stride, scale2, nmesh, tw, st)));
    return 0;
}

int pm_fft_c2r_x3(int log2n, const float2* in, long long comp_stride, long long slot_stride, float4* out,
                  long long out_stride, int nmesh, const float2* tw, cudaStream_t st) {
    PM_DISPATCH_LOG2N(log2n, (launch_x_c2r3<LG>(in, comp_stride, slot_stride, out, out_stride, nmesh, tw, st)));
    return 0;
}

int pm_fft_y(int log2n, float2* data, long long stride, int nmesh, int dir, const float2* tw, cudaStream_t st) {
    PM_DISPATCH_LOG2N(log2n, (launch_y<LG>(data, stride, nmesh, dir, tw, st)));
    return 0;
}

int pm_fft_z(int log2n, int mode, const PmZPass& p, int nslots, cudaStream_t st) {
    ZArgs a;
    for (int i = 0; i < 3; ++i) a.in[i] = p.in[i];
    for (int i = 0; i < 6; ++i) a.out[i] = p.out[i];
    a.slot_stride = p.slot_stride;
    a.tw = p.tw;
    a.lap1 = p.lap1;
    a.grad1 = p.grad1;
    a.dec1 = p.dec1;
    a.ictab = p.ictab;
    a.pk_out = p.pk_out;
    a.nbins = p.nbins;
    a.scale = p.scale;
    a.kf = p.kf;
    PM_DISPATCH_LOG2N(log2n, (launch_z<LG>(mode, a, nslots, st)));
    return 0;
}
