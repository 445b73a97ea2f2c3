// Power spectrum for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a host
// callback or a CUDA-graph-driven pipeline that forbids allocations, plugins
// whose host application owns every device allocation, or processes running
// under a fixed device-memory budget that is already committed.  For them this
// file offers one entry point, pm_power_spectrum_static, that needs no handle
// and allocates nothing: its scratch (density mesh, half spectrum, twiddles
// and FP64 bin sums) lives in one file-scope __device__ array of
// fixed size, which every GPU that loads the library holds until the process
// exits.  The kernels are the same deposit / FFT / binning kernels the
// handle-based pm_power_spectrum launches.
#include <cmath>
#include <mutex>

#include "../../include/pmgb.h"
#include "pm_kernels.h"

namespace {

constexpr int kMaxMesh = PM_STATIC_PK_MAX_MESH;
constexpr int kMaxBins = PM_STATIC_PK_MAX_MESH / 2;
constexpr long long kMeshFloats = (long long)kMaxMesh * kMaxMesh * kMaxMesh;
constexpr long long kSpecCplx = (long long)kMaxMesh * kMaxMesh * (kMaxMesh / 2 + SPEC_PAD);

// byte offsets inside the scratch array (each 256-byte aligned); the FP64 bin
// accumulators hold sum w |rho^|^2 per bin
constexpr long long align256(long long b) { return (b + 255) / 256 * 256; }
constexpr long long kOffRho = 0;
constexpr long long kOffSpec = align256(kOffRho + 4 * kMeshFloats);
constexpr long long kOffTw = align256(kOffSpec + 8 * kSpecCplx);
constexpr long long kOffAcc = align256(kOffTw + 8 * kMaxMesh);
constexpr long long kOffCoef = align256(kOffAcc + 8 * kMaxBins);
constexpr long long kScratchBytes = align256(kOffCoef + (long long)sizeof(SlotCoef));

static __device__ __align__(256) unsigned char g_pk_scratch[kScratchBytes];

// device address of g_pk_scratch per device, set up once per device
std::mutex g_mu;
void* g_addr[64] = {};

// twiddles exp(-2 pi i m / n) and the unit coefficient
__global__ void k_static_tables(float2* tw, int n, SlotCoef* coef) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * m / n, &s, &c);
        tw[m] = make_float2((float)c, (float)-s);
        if (m == 0) {
            SlotCoef u{};
            u.active = 1;
            *coef = u;
        }
    }
}

int ilog2s(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

}  // namespace

extern "C" int pm_power_spectrum_static(const float* disp, int32_t n_part, double box, int32_t n_mesh,
                                        int32_t n_bins, void* stream, double* k, double* pk, int64_t* n_modes) {
    const bool p2 = n_part >= 16 && n_part <= 1024 && (n_part & (n_part - 1)) == 0;
    const bool m2 = n_mesh >= 16 && n_mesh <= kMaxMesh && (n_mesh & (n_mesh - 1)) == 0;
    if (!disp || !k || !pk || !n_modes || !p2 || !(box > 0)) return PM_ERR_ARG;
    if (!m2) return PM_ERR_ARG;                               // larger meshes need the handle API
    if (n_bins < 1 || n_bins > n_mesh / 2) return PM_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PM_ERR_CUDA;
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            // host code only sees a host-side stand-in for g_pk_scratch: ask the runtime for the
            // device address on this device (once per device; do it before any stream capture)
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_pk_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return PM_ERR_CUDA;
            }
            g_addr[dev] = p;
        }
        base = g_addr[dev];
    }
    unsigned char* s = static_cast<unsigned char*>(base);
    float* rho = reinterpret_cast<float*>(s + kOffRho);
    float2* spec = reinterpret_cast<float2*>(s + kOffSpec);
    float2* tw = reinterpret_cast<float2*>(s + kOffTw);
    double* acc = reinterpret_cast<double*>(s + kOffAcc);
    SlotCoef* coef = reinterpret_cast<SlotCoef*>(s + kOffCoef);

    cudaStream_t st = (cudaStream_t)stream;
    const int n = n_mesh, l2 = ilog2s(n);
    const long long M = (long long)n * n * n;
    const long long S = (long long)n * n * (n / 2 + SPEC_PAD);
    // the array keeps the previous call's contents: clear what accumulates
    cudaMemsetAsync(rho, 0, sizeof(float) * M, st);
    cudaMemsetAsync(spec, 0, sizeof(float2) * S, st);
    cudaMemsetAsync(acc, 0, sizeof(double) * n_bins, st);
    k_static_tables<<<(n + 255) / 256, 256, 0, st>>>(tw, n, coef);
    PmGeom g;
    g.log2np = ilog2s(n_part);
    g.log2ng = l2;
    g.inv_h = (float)(n / box);
    g.slot_part = 3ll * n_part * n_part * n_part;
    g.slot_mesh = M;
    pm_deposit(2, g, disp, nullptr, coef, 0, 0.f, rho, 1, st);
    pm_fft_r2c_x(l2, rho, M, spec, S, 1, tw, st);
    pm_fft_y(l2, spec, S, 1, -1, tw, st);
    PmZPass z{};
    z.in[0] = spec;
    z.slot_stride = S;
    z.tw = tw;
    z.pk_out = acc;
    z.nbins = n_bins;
    pm_fft_z(l2, PM_Z_PK, z, 1, st);
    double h_acc[kMaxBins];
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h_acc, acc, sizeof(double) * n_bins, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return PM_ERR_CUDA;
    }
    // exact mode counts and |m| sums of each bin (full n^3 grid through the half spectrum)
    double cnt[kMaxBins] = {}, ksum[kMaxBins] = {};
    for (int kx = 0; kx <= n / 2; ++kx) {
        const double w = (kx == 0 || kx == n / 2) ? 1.0 : 2.0;
        for (int y = 0; y < n; ++y) {
            const int my = y < n / 2 ? y : y - n;
            for (int zz = 0; zz < n; ++zz) {
                const int mz = zz < n / 2 ? zz : zz - n;
                const int sq = kx * kx + my * my + mz * mz;
                const int b = (int)std::floor(std::sqrt((double)sq) - 0.5);
                if (sq == 0 || b < 0 || b >= n_bins) continue;
                cnt[b] += w;
                ksum[b] += w * std::sqrt((double)sq);
            }
        }
    }
    const double N = (double)n_part * n_part * n_part;
    const double kf = 2.0 * M_PI / box, MN = (double)M / N;
    for (int i = 0; i < n_bins; ++i) {
        n_modes[i] = (int64_t)std::llround(cnt[i]);
        k[i] = cnt[i] > 0 ? ksum[i] / cnt[i] * kf : 0.0;
        pk[i] = cnt[i] > 0 ? h_acc[i] / cnt[i] * MN * MN * box * box * box / ((double)M * (double)M) : 0.0;
    }
    return PM_OK;
}
