// Batched shared-memory FFT used by every spectral pass of the PM solver
// (Sec. 2.5: real FFT of the density, Poisson/gradient kernels, inverse FFTs).
//
// Self-sorting (Stockham) iteration, radix 8 with one closing radix-2 or
// radix-4 stage when log2 N is not a multiple of 3.  A stage of radix R with
// Ns = product of the earlier radices takes, for butterfly jj in [0, N/R),
// v[r] = x[jj + r N/R], multiplies v[r] by w^(r (jj mod Ns)), w = exp(s 2 pi i /(Ns R)),
// applies an R-point DFT and stores v[r] at (jj / Ns) Ns R + (jj mod Ns) + r Ns.
// The output comes out in natural order.
//
// NL independent lines live in shared memory; element e of line l is at
// s[l * LS + e * ES].  Each of the NL * N / 8 threads owns eight elements of
// one line in every stage (one radix-8, two radix-4 or four radix-2
// butterflies), line = tid % NL, so consecutive threads touch consecutive
// lines: row tiles use an odd line stride LS and column tiles ES = NL, both
// bank-conflict free.  The stages work in place with a barrier between the
// loads and the stores.
#pragma once
#include "pm_common.cuh"

namespace pmfft {

constexpr float kS = 0.70710678118654752440f;   // 1/sqrt(2)

template <int DIR>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
    float2 t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
    // X0 = x0+x1+x2+x3, X1 = x0 + s x1 - x2 - s x3 with s = exp(DIR i pi/2) = DIR i, ...
    float2 t0 = cadd(x0, x2), t1 = csub(x0, x2);
    float2 t2 = cadd(x1, x3), t3 = cmul_i(csub(x1, x3), DIR);
    x0 = cadd(t0, t2);
    x2 = csub(t0, t2);
    x1 = cadd(t1, t3);
    x3 = csub(t1, t3);
}

template <int DIR>
__device__ __forceinline__ void dft8(float2* v) {
    // split into even/odd halves: a_r = v_r + v_{r+4}, b_r = (v_r - v_{r+4}) w8^r
    float2 a0 = cadd(v[0], v[4]), b0 = csub(v[0], v[4]);
    float2 a1 = cadd(v[1], v[5]), b1 = csub(v[1], v[5]);
    float2 a2 = cadd(v[2], v[6]), b2 = csub(v[2], v[6]);
    float2 a3 = cadd(v[3], v[7]), b3 = csub(v[3], v[7]);
    // w8 = exp(DIR i pi / 4) = (1 + DIR i)/sqrt2 ; w8^2 = DIR i ; w8^3 = (-1 + DIR i)/sqrt2
    b1 = make_float2(kS * (b1.x - DIR * b1.y), kS * (b1.y + DIR * b1.x));
    b2 = cmul_i(b2, DIR);
    b3 = make_float2(kS * (-b3.x - DIR * b3.y), kS * (-b3.y + DIR * b3.x));
    dft4<DIR>(a0, a1, a2, a3);
    dft4<DIR>(b0, b1, b2, b3);
    v[0] = a0; v[2] = a1; v[4] = a2; v[6] = a3;
    v[1] = b0; v[3] = b1; v[5] = b2; v[7] = b3;
}

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

// twiddle exp(DIR * 2 pi i * m / TWN) from a table of exp(-2 pi i m / TWN)
template <int DIR>
__device__ __forceinline__ float2 twiddle(const float2* tw, int m) {
    float2 w = tw[m];
    return DIR < 0 ? w : cconj(w);
}

// One Stockham stage of radix R (R in {2, 4, 8}), Ns = product of earlier radices.
template <int N, int R, int NS, int NL, int LS, int ES, int DIR>
__device__ __forceinline__ void stage(float2* s, const float2* tw, int twstride, bool active) {
    constexpr int NB = 8 / R;               // butterflies per thread
    const int tid = threadIdx.x;
    const int line = tid % NL;
    const int j = tid / NL;                 // in [0, N/8)
    float2 v[8];
    float2* base = s + line * LS;
    if (active) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int jj = j + b * (N / 8);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = base[(jj + r * (N / R)) * ES];
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const int jj = j + b * (N / 8);
        const int k = jj % NS;
        float2* vb = v + b * R;
        if (NS > 1) {
            // w^(r k) with w = exp(DIR 2 pi i / (NS R)): table index r k N/(NS R) * twstride
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const int m = (r * k * (N / (NS * R))) * twstride;
                vb[r] = cmul(vb[r], twiddle<DIR>(tw, m));
            }
        }
        if (R == 8) dft8<DIR>(vb);
        if (R == 4) dft4<DIR>(vb[0], vb[1], vb[2], vb[3]);
        if (R == 2) dft2<DIR>(vb[0], vb[1]);
        const int o = (jj / NS) * NS * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) base[(o + r * NS) * ES] = vb[r];
    }
    }
    __syncthreads();
}

// Full N-point transform of NL lines in shared memory (caller syncs before).
// Every thread of the block must call it (it contains barriers); threads with
// index >= NL * N / 8 only join the barriers.
template <int N, int NL, int LS, int ES, int DIR>
__device__ __forceinline__ void fft_lines(float2* s, const float2* tw, int twstride) {
    static_assert(N >= 8 && (N & (N - 1)) == 0, "N must be a power of two >= 8");
    constexpr int L2 = ilog2(N);
    constexpr int N8 = L2 / 3;              // radix-8 stages
    constexpr int REM = 1 << (L2 - 3 * N8); // closing radix (1 = none)
    const bool active = threadIdx.x < NL * N / 8;
    if constexpr (N8 >= 1) stage<N, 8, 1, NL, LS, ES, DIR>(s, tw, twstride, active);
    if constexpr (N8 >= 2) stage<N, 8, 8, NL, LS, ES, DIR>(s, tw, twstride, active);
    if constexpr (N8 >= 3) stage<N, 8, 64, NL, LS, ES, DIR>(s, tw, twstride, active);
    if constexpr (N8 >= 4) stage<N, 8, 512, NL, LS, ES, DIR>(s, tw, twstride, active);
    constexpr int NSR = 1 << (3 * N8);
    if constexpr (REM == 4) stage<N, 4, NSR, NL, LS, ES, DIR>(s, tw, twstride, active);
    if constexpr (REM == 2) stage<N, 2, NSR, NL, LS, ES, DIR>(s, tw, twstride, active);
}


// ---------------------------------------------------------------------------
// Functor form: the first stage reads its inputs through `ld(line, e)` and the
// last stage writes through `st(line, e, v)`, so a transform can start from
// global memory (or another tile, with an elementwise multiplier applied on the
// fly) and end in global memory without an extra shared-memory round trip.
// Middle stages work in place on the shared-memory tile `sm`.

// The loads of one stage: thread (line, j) takes v[b R + r] = element j + b N/8 + r N/R.
template <int N, int R, int NL, class Ld>
__device__ __forceinline__ void stage_load(const Ld& ld, float2 v[8], bool active) {
    constexpr int NB = 8 / R;
    const int line = threadIdx.x % NL;
    const int j = threadIdx.x / NL;
    if (active) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int jj = j + b * (N / 8);
#pragma unroll
            for (int r = 0; r < R; ++r) v[b * R + r] = ld(line, jj + r * (N / R));
        }
    }
}

// The twiddles, butterflies and stores of one stage on loaded values v (STORE =
// false: the results stay in v, butterfly b's outputs r at v[b R + r]).
template <int N, int R, int NS, int NL, int DIR, class St, bool STORE = true>
__device__ __forceinline__ void stage_cs(float2 v[8], const St& st, const float2* tw, int twstride, bool active) {
    constexpr int NB = 8 / R;
    const int line = threadIdx.x % NL;
    const int j = threadIdx.x / NL;
    if (active) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int jj = j + b * (N / 8);
            const int k = jj % NS;
            float2* vb = v + b * R;
            if (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) vb[r] = cmul(vb[r], twiddle<DIR>(tw, (r * k * (N / (NS * R))) * twstride));
            }
            if (R == 8) dft8<DIR>(vb);
            if (R == 4) dft4<DIR>(vb[0], vb[1], vb[2], vb[3]);
            if (R == 2) dft2<DIR>(vb[0], vb[1]);
            if (STORE) {
                const int o = (jj / NS) * NS * R + k;
#pragma unroll
                for (int r = 0; r < R; ++r) st(line, o + r * NS, vb[r]);
            }
        }
    }
}

template <int N, int R, int NS, int NL, int DIR, bool MIDSYNC, class Ld, class St>
__device__ __forceinline__ void stage_io(const Ld& ld, const St& st, const float2* tw, int twstride, bool active) {
    float2 v[8];
    stage_load<N, R, NL>(ld, v, active);
    if (MIDSYNC) __syncthreads();
    stage_cs<N, R, NS, NL, DIR>(v, st, tw, twstride, active);
}

// radix of stage i (0-based) and Ns before it for an N-point transform
template <int N>
struct Plan {
    static constexpr int L2 = ilog2(N);
    static constexpr int N8 = L2 / 3;
    static constexpr int REM = 1 << (L2 - 3 * N8);
    static constexpr int S = N8 + (REM > 1 ? 1 : 0);
    __host__ __device__ static constexpr int radix(int i) { return i < N8 ? 8 : REM; }
    __host__ __device__ static constexpr int ns(int i) { return 1 << (3 * (i < N8 ? i : N8)); }
};

// Full transform: ld -> (stage 0) -> sm -> ... -> (last stage) -> st.
// FIRST_SYNC: stage 0 reads from `sm` itself (in-place first stage).
// LAST_SMEM:  st writes into `sm` (in-place last stage).
// The caller guarantees `sm` may be overwritten on entry (barrier before) and
// synchronises after if st wrote shared memory that others read.
template <int N, int NL, int DIR, bool FIRST_SYNC, bool LAST_SMEM, class Ld, class St, class Sm>
__device__ __forceinline__ void fft_io(const Ld& ld, const St& st, const Sm& sm, const float2* tw, int twstride) {
    using Pl = Plan<N>;
    static_assert(Pl::S >= 2, "N must have at least two stages");
    const bool active = threadIdx.x < NL * N / 8;
    stage_io<N, Pl::radix(0), 1, NL, DIR, FIRST_SYNC>(ld, sm, tw, twstride, active);
    __syncthreads();
    if constexpr (Pl::S > 2) {
        stage_io<N, Pl::radix(1), Pl::ns(1), NL, DIR, true>(sm, sm, tw, twstride, active);
        __syncthreads();
    }
    if constexpr (Pl::S > 3) {
        stage_io<N, Pl::radix(2), Pl::ns(2), NL, DIR, true>(sm, sm, tw, twstride, active);
        __syncthreads();
    }
    static_assert(Pl::S <= 4, "at most 4 stages (N <= 4096)");
    stage_io<N, Pl::radix(Pl::S - 1), Pl::ns(Pl::S - 1), NL, DIR, LAST_SMEM>(sm, st, tw, twstride, active);
}

// First-stage inputs of fft_pre (the loads fft_io's first stage makes), so that a
// caller can have the next transform's loads in flight during the current one.
template <int N, int NL, class Ld>
__device__ __forceinline__ void fft_first_load(const Ld& ld, float2 v[8]) {
    stage_load<N, Plan<N>::radix(0), NL>(ld, v, threadIdx.x < NL * N / 8);
}

// fft_io from first-stage inputs already in registers.  The first stage writes
// `sm`, so the caller puts a barrier between any earlier reader of `sm` and this.
template <int N, int NL, int DIR, bool LAST_SMEM, class St, class Sm>
__device__ __forceinline__ void fft_pre(float2 v[8], const St& st, const Sm& sm, const float2* tw, int twstride) {
    using Pl = Plan<N>;
    static_assert(Pl::S >= 2, "N must have at least two stages");
    const bool active = threadIdx.x < NL * N / 8;
    stage_cs<N, Pl::radix(0), 1, NL, DIR>(v, sm, tw, twstride, active);
    __syncthreads();
    if constexpr (Pl::S > 2) {
        stage_io<N, Pl::radix(1), Pl::ns(1), NL, DIR, true>(sm, sm, tw, twstride, active);
        __syncthreads();
    }
    if constexpr (Pl::S > 3) {
        stage_io<N, Pl::radix(2), Pl::ns(2), NL, DIR, true>(sm, sm, tw, twstride, active);
        __syncthreads();
    }
    stage_io<N, Pl::radix(Pl::S - 1), Pl::ns(Pl::S - 1), NL, DIR, LAST_SMEM>(sm, st, tw, twstride, active);
}

// All stages but the last of an N-point transform: the first reads `ld`, the
// others work in place on `sm`; ends with a barrier, the data in `sm`.
template <int N, int NL, int DIR, class Ld, class Sm>
__device__ __forceinline__ void fft_head(const Ld& ld, const Sm& sm, const float2* tw, int twstride) {
    using Pl = Plan<N>;
    const bool active = threadIdx.x < NL * N / 8;
    stage_io<N, Pl::radix(0), 1, NL, DIR, false>(ld, sm, tw, twstride, active);
    __syncthreads();
    if constexpr (Pl::S > 2) {
        stage_io<N, Pl::radix(1), Pl::ns(1), NL, DIR, true>(sm, sm, tw, twstride, active);
        __syncthreads();
    }
    if constexpr (Pl::S > 3) {
        stage_io<N, Pl::radix(2), Pl::ns(2), NL, DIR, true>(sm, sm, tw, twstride, active);
        __syncthreads();
    }
}

// The last stage after fft_head, into registers: out[r'] = element j + r' N/8 of
// line l (thread = (l, j) = (tid % NL, tid / NL)), the order in which the first
// stage of another transform (fft_pre) takes its inputs.  The last stage of
// radix R leaves butterfly b's output r at element j + b N/8 + r N/R, i.e. r' =
// b + r 8/R.
template <int N, int NL, int DIR, class Sm>
__device__ __forceinline__ void fft_tail_regs(const Sm& sm, float2 out[8], const float2* tw, int twstride) {
    using Pl = Plan<N>;
    constexpr int R = Pl::radix(Pl::S - 1), NS = Pl::ns(Pl::S - 1), NB = 8 / R;
    static_assert(NS * R == N, "last stage");
    const bool active = threadIdx.x < NL * N / 8;
    float2 v[8];
    stage_load<N, R, NL>(sm, v, active);
    stage_cs<N, R, NS, NL, DIR, Sm, false>(v, sm, tw, twstride, active);
#pragma unroll
    for (int b = 0; b < NB; ++b)
#pragma unroll
        for (int r = 0; r < R; ++r) out[b + r * NB] = v[b * R + r];
}

// Shared-memory column tile of NL = COL_TILE columns: element e of column l at
// (e + e / 8) * NL + l (one padding row every 8 rows keeps the radix-8 first
// stage's stores free of bank conflicts).
struct ColTile {
    float2* s;
    __device__ __forceinline__ int at(int l, int e) const { return (e + (e >> 3)) * COL_TILE + l; }
    __device__ __forceinline__ float2 operator()(int l, int e) const { return s[at(l, e)]; }
    __device__ __forceinline__ void operator()(int l, int e, float2 v) const { s[at(l, e)] = v; }
};
__host__ __device__ constexpr int col_tile_elems(int n) { return (n + n / 8) * COL_TILE; }

// Global column tile: element e of column l at g[e * es + l]
struct GCols {
    float2* g;
    long long es;
    __device__ __forceinline__ float2 operator()(int l, int e) const { return g[e * es + l]; }
    __device__ __forceinline__ void operator()(int l, int e, float2 v) const { g[e * es + l] = v; }
};

}  // namespace pmfft
