// C ABI of libpmgb (include/pmgb.h): handle, workspace, tables and the
// orchestration of the PM step (Sec. 2.4 Eq. dkd, Sec. 2.5) on one GPU.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/pmgb.h"
#include "cosmo_host.h"
#include "pm_kernels.h"

#define PM_NPHASE 12

namespace {

thread_local std::string g_init_error;

int ilog2i(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}
bool pow2_in_range(int n) { return n >= 16 && n <= 1024 && (n & (n - 1)) == 0; }
long long spec_elems(int n) { return (long long)n * n * spec_pitch(n); }   // complex per spectrum
long long mesh_elems(int n) { return (long long)n * n * n; }

// elementwise x = a * x + b over count floats
__global__ void k_affine(float* x, long long count, float a, float b) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) x[i] = a * x[i] + b;
}

}  // namespace

struct pm_handle {
    pm_config cfg{};
    cudaStream_t stream = nullptr;
    int B = 1, np = 0, ng = 0, npk = 0, nmax = 0;
    int ngrids = 1, ncomp = 3;
    int mak = 2;                 // mass assignment kernel of deposit and interpolation (5 = ES, NUFFT)
    std::unique_ptr<pmcosmo::Growth> growth;
    std::vector<pmcosmo::StepCoef> table;
    std::string err;

    // device workspace
    float* rho = nullptr;        // [B][ngrids][max(Mg, Mpk)]
    float2* spec = nullptr;      // [B][ncomp][spec_elems(nmax)]
    float4* force = nullptr;     // [B][ngrids][Mg] interleaved (gx, gy, gz, 0)
    SlotCoef* d_table = nullptr; // [n_steps]
    SlotCoef* d_slots = nullptr; // [B]
    SlotCoef* d_unit = nullptr;  // active, tau1 = 0
    float2* d_tw[11] = {};       // twiddles exp(-2 pi i m / 2^l)
    float* d_lap = nullptr;      // [ng]
    float* d_grad = nullptr;     // [ng]
    float* d_dec = nullptr;      // [ng] deconvolution 1 / W^(k)^2 per axis, NULL when off
    float* d_ictab = nullptr;    // [3 (np/2)^2 + 1]
    double* d_pk = nullptr;      // [B][pk_bins_cap]: sum over each bin of w |rho^|^2
    int pk_bins_cap = 0;
    struct BinTable {
        std::vector<double> count, ksum;            // exact per-bin mode counts and sum |m|
    };
    std::map<std::pair<int, int>, BinTable> bintabs;   // (n, nbins)
    // slot mode
    SlotCoef* h_slots = nullptr; // pinned ring [4][B]
    cudaEvent_t slot_ev[4] = {};
    int slot_ring = 0;
    std::map<int, std::vector<pmcosmo::StepCoef>> tables_by_nsteps;
    // adjoint scratch: 3 meshes per slot of max(Mg, Np) floats (allocated on first use)
    float* adj3 = nullptr;
    float* jrho = nullptr;       // forward mode: tangent density [B][rho_slot]
    float4* jforce = nullptr;    // forward mode: tangent force mesh [B][Mg]
    double* d_dot = nullptr;
    // host-buffer mode
    float *d_noise = nullptr, *d_disp = nullptr, *d_vel = nullptr;
    size_t bytes = 0;
    // optional per-phase timing with CUDA events on the handle's stream
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_marks;   // (phase, index of start event; end = +1)
    int64_t launches[PM_NPHASE] = {};
    int cur_phase = -1, cur_ev = -1;
    void phase(int p, int nlaunch) {
        launches[p] += nlaunch;
        if (!prof) return;
        if (ev_pool.size() < ev_marks.size() * 2 + 2) {
            for (int i = 0; i < 64; ++i) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                ev_pool.push_back(e);
            }
        }
        const int idx = (int)ev_marks.size() * 2;
        cudaEventRecord(ev_pool[idx], stream);
        ev_marks.push_back({p, idx});
    }
    void phase_end() {
        if (!prof || ev_marks.empty()) return;
        cudaEventRecord(ev_pool[ev_marks.back().second + 1], stream);
    }

    long long Mg() const { return mesh_elems(ng); }
    long long Np() const { return mesh_elems(np); }
    long long rho_slot() const { return (long long)ngrids * std::max(mesh_elems(ng), mesh_elems(npk)); }
    long long spec_slot() const { return (long long)ncomp * spec_elems(nmax); }
    int force_mode() const { return ngrids == 2 ? PM_Z_FORCE_IL : PM_Z_FORCE; }

    int fail(int code, const char* fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }
    int check_launch(const char* what) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(PM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
        return PM_OK;
    }
};

namespace {

SlotCoef to_slot(const pmcosmo::StepCoef& c) {
    SlotCoef s{};
    s.tau1 = (float)c.tau1;
    s.tau2 = (float)c.tau2;
    s.alpha = (float)c.alpha;
    s.kick = (float)(c.beta / (c.D_half * c.D_half));   // A = g / D_half^2
    s.active = 1;
    return s;
}

// Table 2 kernels in physical units (H = cell size): gradient (imaginary part)
// and second derivative of a 1D stencil as functions of k.
double grad1d(double k, double H, int order) {
    const double x = k * H;
    switch (order) {
        case 0: return k;
        case 2: return std::sin(x) / H;
        case 4: return (8.0 * std::sin(x) - std::sin(2.0 * x)) / (6.0 * H);
        case 6: return (45.0 * std::sin(x) - 9.0 * std::sin(2.0 * x) + std::sin(3.0 * x)) / (30.0 * H);
    }
    return 0.0;
}
double lap1d(double k, double H, int order) {
    const double x = k * H;
    switch (order) {
        case 0: return -k * k;
        case 2: return -2.0 * (1.0 - std::cos(x)) / (H * H);
        case 4: return -(std::cos(2.0 * x) - 16.0 * std::cos(x) + 15.0) / (6.0 * H * H);
        case 6: return -(-2.0 * std::cos(3.0 * x) + 27.0 * std::cos(2.0 * x) - 270.0 * std::cos(x) + 245.0) / (90.0 * H * H);
    }
    return 0.0;
}

int validate(const pm_config* c, std::string& why) {
    char buf[256];
    auto bad = [&](const char* m) { why = m; return PM_ERR_ARG; };
    if (!c) return bad("config is NULL");
    if (!pow2_in_range(c->n_part)) return bad("n_part must be a power of two in [16, 1024]");
    if (!pow2_in_range(c->n_mesh)) return bad("n_mesh must be a power of two in [16, 1024]");
    if (c->pk_mesh_max && !pow2_in_range(c->pk_mesh_max)) return bad("pk_mesh_max must be 0 or a power of two in [16, 1024]");
    if (!(c->box > 0)) return bad("box must be > 0");
    if (c->order < 2 || c->order > 4) return bad("order must be 2 (CIC), 3 (TSC) or 4 (PCS)");
    if (c->interlace != 0 && c->interlace != 1) return bad("interlace must be 0 or 1");
    if (c->deconvolve != 0 && c->deconvolve != 1) return bad("deconvolve must be 0 or 1");
    if (c->lpt_order < 0 || c->lpt_order > 2) return bad("lpt_order must be 0, 1 (Zel'dovich) or 2 (2LPT)");
    if (c->nufft != 0 && c->nufft != 1) return bad("nufft must be 0 or 1");
    if (c->nufft) {
        if (c->grad_order != 0 || c->lap_order != 0) return bad("nufft needs the exact kernels (grad_order = lap_order = 0)");
        if (c->interlace || c->deconvolve) return bad("nufft excludes interlace and deconvolve");
        if (2 * c->n_mesh > 1024) return bad("nufft: the upsampled grid 2 n_mesh must be <= 1024");
    }
    for (int o : {c->grad_order, c->lap_order})
        if (o != 0 && o != 2 && o != 4 && o != 6) return bad("grad_order / lap_order must be 0, 2, 4 or 6");
    if (!(c->omega_m > 0 && c->omega_m <= 1)) return bad("omega_m must be in (0, 1]");
    if (!(c->h > 0) || !(c->sigma8 > 0)) return bad("h and sigma8 must be > 0");
    if (!(c->a_ini > 1e-4 && c->a_end > c->a_ini && c->a_end <= 3.0)) return bad("need 1e-4 < a_ini < a_end <= 3");
    if (c->n_steps < 1 || c->n_steps > 100000) return bad("n_steps must be in [1, 100000]");
    if (c->stepper != 0 && c->stepper != 1) return bad("stepper must be 0 (BullFrog) or 1 (FastPM)");
    if (c->time_var != 0 && c->time_var != 1) return bad("time_var must be 0 (D) or 1 (a)");
    if (c->batch < 1 || c->batch > 4096) return bad("batch must be in [1, 4096]");
    const double Np = (double)c->n_part * c->n_part * c->n_part;
    if (Np * c->batch > 2.0e9) {
        snprintf(buf, sizeof buf, "batch * n_part^3 = %.3g exceeds 2e9 particles", Np * c->batch);
        why = buf;
        return PM_ERR_ARG;
    }
    return PM_OK;
}

size_t workspace_bytes(const pm_config* c) {
    const int ng = c->nufft ? 2 * c->n_mesh : c->n_mesh, np = c->n_part;
    const int npk = c->pk_mesh_max ? c->pk_mesh_max : c->n_mesh;
    const int nmax = std::max(ng, std::max(np, npk));
    const int ngrids = c->interlace ? 2 : 1, ncomp = c->interlace ? 6 : 3;
    size_t b = 0;
    b += (size_t)c->batch * ngrids * std::max(mesh_elems(ng), mesh_elems(npk)) * 4;
    b += (size_t)c->batch * ncomp * spec_elems(nmax) * 8;
    // force meshes (float4); 2LPT ICs also use them for four real lattice fields per slot
    b += (size_t)c->batch * std::max((long long)ngrids * mesh_elems(ng),
                                     c->lpt_order == 2 ? (long long)mesh_elems(np) : 0ll) * 16;
    b += (size_t)(3 * (np / 2) * (np / 2) + 1) * 4 + 8 * 1024 * 8 * 2 + (size_t)ng * 8;
    b += (size_t)(c->n_steps + c->batch + 1) * sizeof(SlotCoef);
    return b;
}

template <typename T>
int dalloc(pm_handle* h, T** p, size_t count, const char* what) {
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return h->fail(PM_ERR_OOM, "cudaMalloc(%s, %zu bytes): %s", what, count * sizeof(T), cudaGetErrorString(e));
    }
    h->bytes += count * sizeof(T);
    return PM_OK;
}

int upload_twiddles(pm_handle* h, int n) {
    const int l = ilog2i(n);
    if (h->d_tw[l]) return PM_OK;
    std::vector<float2> tw(n);
    for (int m = 0; m < n; ++m) {
        const double ang = 2.0 * M_PI * m / n;
        tw[m] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    int rc = dalloc(h, &h->d_tw[l], n, "twiddles");
    if (rc) return rc;
    if (cudaMemcpy(h->d_tw[l], tw.data(), n * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
        return h->fail(PM_ERR_CUDA, "upload twiddles");
    return PM_OK;
}

PmGeom geom(const pm_handle* h, int nmesh, long long slot_mesh) {
    PmGeom g;
    g.log2np = ilog2i(h->np);
    g.log2ng = ilog2i(nmesh);
    g.inv_h = (float)(nmesh / h->cfg.box);
    g.slot_part = 3 * h->Np();
    g.slot_mesh = slot_mesh;
    return g;
}

// Forward real FFT of ngrids density meshes per slot (rho, slot stride rho_slot)
// into spectra comp 0..ngrids-1; then the fused z pass producing ncomp spectra.
int spectral_force(pm_handle* h, const float* src, long long src_slot, long long src_grid, float scale,
                   float* force_out, float4* force4, int nslots, int clear_src = 0) {
    const int n = h->ng, l2 = ilog2i(n);
    const long long S = spec_elems(n), SS = (long long)h->ncomp * S;
    cudaStream_t st = h->stream;
    h->phase(1, h->ngrids);
    for (int g = 0; g < h->ngrids; ++g)
        if (pm_fft_r2c_x(l2, src + g * src_grid, src_slot, h->spec + g * S, SS, nslots, h->d_tw[l2], st, clear_src))
            return h->fail(PM_ERR_ARG, "unsupported mesh size %d", n);
    h->phase_end();
    h->phase(2, h->ngrids);
    for (int g = 0; g < h->ngrids; ++g) pm_fft_y(l2, h->spec + g * S, SS, nslots, -1, h->d_tw[l2], st);
    h->phase_end();
    PmZPass z{};
    z.in[0] = h->spec;
    z.in[1] = h->spec + S;
    z.slot_stride = SS;
    z.tw = h->d_tw[l2];
    z.lap1 = h->d_lap;
    z.grad1 = h->d_grad;
    z.dec1 = h->d_dec;
    z.scale = scale;
    z.kf = (float)(2.0 * M_PI / h->cfg.box);
    const int go = h->cfg.grad_order;
    if (force4 && go != 0) {
        // finite-difference gradient: one potential per grid, inverse transformed once,
        // then g = -D1 phi as a real-space stencil (the same operator as D1(k) in k space)
        for (int g = 0; g < h->ngrids; ++g) z.out[g] = h->spec + g * S;
        h->phase(3, 1);
        pm_fft_z(l2, h->ngrids == 2 ? PM_Z_POT_IL : PM_Z_POT, z, nslots, st);
        h->phase_end();
        h->phase(4, h->ngrids);
        for (int g = 0; g < h->ngrids; ++g) pm_fft_y(l2, h->spec + g * S, SS, nslots, 1, h->d_tw[l2], st);
        h->phase_end();
        // the real potential of grid g goes to the unused spectrum slot ngrids + g (a
        // spectrum slot holds more than n^3 floats), so the density mesh stays as the
        // forward x pass left it
        auto phi = [&](int g) { return reinterpret_cast<float*>(h->spec + (h->ngrids + g) * S); };
        h->phase(5, h->ngrids);
        for (int g = 0; g < h->ngrids; ++g)
            pm_fft_c2r_x(l2, h->spec + g * S, SS, phi(g), 2 * SS, nullptr, 0, 0.f, nslots, h->d_tw[l2], st);
        h->phase_end();
        h->phase(11, h->ngrids);
        for (int g = 0; g < h->ngrids; ++g)
            pm_grad_stencil(go, l2, (float)(n / h->cfg.box), phi(g), 2 * SS, force4 + g * h->Mg(),
                            (long long)h->ngrids * h->Mg(), nslots, st);
        h->phase_end();
        return h->check_launch("force spectral passes");
    }
    for (int c = 0; c < h->ncomp; ++c) z.out[c] = h->spec + c * S;
    h->phase(3, 1);
    pm_fft_z(l2, h->force_mode(), z, nslots, st);
    h->phase_end();
    h->phase(4, 1);
    pm_fft_y(l2, h->spec, S, nslots * h->ncomp, 1, h->d_tw[l2], st);
    h->phase_end();
    h->phase(5, force4 ? h->ngrids : 1);
    if (force4) {
        for (int g = 0; g < h->ngrids; ++g)
            pm_fft_c2r_x3(l2, h->spec + 3 * g * S, S, SS, force4 + g * h->Mg(), (long long)h->ngrids * h->Mg(), nslots,
                          h->d_tw[l2], st);
    } else {
        pm_fft_c2r_x(l2, h->spec, S, force_out, h->Mg(), nullptr, 0, 0.f, nslots * h->ncomp, h->d_tw[l2], st);
    }
    h->phase_end();
    return h->check_launch("force spectral passes");
}

}  // namespace

namespace {

int one_step(pm_handle* h, float* disp, float* vel, const SlotCoef* coef, int cstride) {
    cudaStream_t st = h->stream;
    const long long Mg = h->Mg();
    if (cudaMemsetAsync(h->rho, 0, sizeof(float) * h->rho_slot() * h->B, st) != cudaSuccess)
        return h->fail(PM_ERR_CUDA, "memset density");
    const PmGeom gd = geom(h, h->ng, h->rho_slot());
    h->phase(0, h->ngrids);
    for (int g = 0; g < h->ngrids; ++g)
        pm_deposit(h->mak, gd, disp, vel, coef, cstride, 0.5f * g, h->rho + g * Mg, h->B, st);
    h->phase_end();
    // delta = rho M/N - 1; the -1 only touches k = 0 (zeroed), and M/N with the
    // 1/M of the inverse transform leaves 1/N on the multiplier
    int rc = spectral_force(h, h->rho, h->rho_slot(), Mg, (float)(1.0 / (double)h->Np()), nullptr, h->force, h->B);
    if (rc) return rc;
    const PmGeom gi = geom(h, h->ng, (long long)h->ngrids * Mg);
    h->phase(6, 1);
    pm_interp_kick(h->mak, h->cfg.interlace, gi, disp, vel, coef, cstride, h->force, h->B, st);
    h->phase_end();
    return h->check_launch("pm step");
}

int bintab_for(pm_handle* h, int n, int nbins, const pm_handle::BinTable** out) {
    auto key = std::make_pair(n, nbins);
    auto it = h->bintabs.find(key);
    if (it != h->bintabs.end()) { *out = &it->second; return PM_OK; }
    // bin floor(|m| - 1/2) of each integer |m|^2 (the z pass takes the same bin in
    // float arithmetic, which is exact for |m|^2 < 2^24)
    const int ns = 3 * (n / 2) * (n / 2) + 1;
    std::vector<int> t(ns);
    for (int s = 0; s < ns; ++s) {
        const int b = (int)std::floor(std::sqrt((double)s) - 0.5);
        t[s] = (s > 0 && b >= 0 && b < nbins) ? b : -1;
    }
    pm_handle::BinTable bt;
    bt.count.assign(nbins, 0.0);
    bt.ksum.assign(nbins, 0.0);
    // modes of the full n^3 grid, counted through the half spectrum kx = 0..n/2
    // (weight 2 for 0 < kx < n/2: the mode and its mirror -k)
    for (int kx = 0; kx <= n / 2; ++kx) {
        const double w = (kx == 0 || kx == n / 2) ? 1.0 : 2.0;
        for (int y = 0; y < n; ++y) {
            const int my = y < n / 2 ? y : y - n;
            for (int z = 0; z < n; ++z) {
                const int mz = z < n / 2 ? z : z - n;
                const int sq = kx * kx + my * my + mz * mz;
                const int b = t[sq];
                if (b < 0) continue;
                bt.count[b] += w;
                bt.ksum[b] += w * std::sqrt((double)sq);
            }
        }
    }
    auto res = h->bintabs.emplace(key, std::move(bt));
    *out = &res.first->second;
    return PM_OK;
}

// One IC spectral chain: forward transform of `src` (slot stride src_stride), the z
// pass `mode` producing three spectra, inverse transforms into three real fields
// per slot at dst (slot stride 3 Np) -- or, for the Zel'dovich pass (dst NULL),
// into vel and D disp.
void ic_chain(pm_handle* h, const float* src, long long src_stride, int mode, float scale, float* dst, float* disp,
              float* vel, int nslots) {
    const int n = h->np, l2 = ilog2i(n);
    const long long S = spec_elems(n), SS = 3 * S;
    cudaStream_t st = h->stream;
    pm_fft_r2c_x(l2, src, src_stride, h->spec, SS, nslots, h->d_tw[l2], st);
    pm_fft_y(l2, h->spec, SS, nslots, -1, h->d_tw[l2], st);
    PmZPass z{};
    z.in[0] = h->spec;
    for (int c = 0; c < 3; ++c) z.out[c] = h->spec + c * S;
    z.slot_stride = SS;
    z.tw = h->d_tw[l2];
    z.ictab = h->d_ictab;
    z.kf = (float)(2.0 * M_PI / h->cfg.box);
    z.scale = scale;
    pm_fft_z(l2, mode, z, nslots, st);
    pm_fft_y(l2, h->spec, S, 3 * nslots, 1, h->d_tw[l2], st);
    if (dst)
        pm_fft_c2r_x(l2, h->spec, S, dst, h->Np(), nullptr, 0, 0.f, 3 * nslots, h->d_tw[l2], st);
    else
        pm_fft_c2r_x(l2, h->spec, S, vel, h->Np(), disp, h->Np(), (float)h->growth->D(h->cfg.a_ini), 3 * nslots,
                     h->d_tw[l2], st);
}

int ic_impl(pm_handle* h, const float* noise, float* disp, float* vel, int nslots) {
    const int n = h->np, l2 = ilog2i(n);
    const long long S = spec_elems(n), SS = 3 * S;
    cudaStream_t st = h->stream;
    if (h->cfg.lpt_order == 2) {
        // 2LPT (Eq. LPT at n = 2): the source L2 = -(3/7) mu_2L from the six second
        // derivatives of psi1 (three at a time into lattice fields t; mu after them,
        // both in the force-mesh buffer), psi2 = Lap^-1 grad L2 into t, then the
        // Zel'dovich state and Psi += D^2 psi2, V += 2 D psi2
        const long long Np = h->Np();
        float* t = reinterpret_cast<float*>(h->force);
        float* mu = t + 3 * Np * nslots;
        h->phase(7, 24);
        ic_chain(h, noise, Np, PM_Z_IC_D2, 0.f, t, nullptr, nullptr, nslots);
        pm_lpt2_source(0, t, mu, Np, nslots, st);
        ic_chain(h, noise, Np, PM_Z_IC_O2, 0.f, t, nullptr, nullptr, nslots);
        pm_lpt2_source(1, t, mu, Np, nslots, st);
        ic_chain(h, mu, Np, PM_Z_LPT2, (float)(1.0 / (double)Np), t, nullptr, nullptr, nslots);
        ic_chain(h, noise, Np, PM_Z_IC, 0.f, nullptr, disp, vel, nslots);
        const double D = h->growth->D(h->cfg.a_ini);
        pm_axpby(disp, disp, t, 1.f, (float)(D * D), 3 * Np * nslots, st);
        pm_axpby(vel, vel, t, 1.f, (float)(2.0 * D), 3 * Np * nslots, st);
        h->phase_end();
        return h->check_launch("2lpt ic");
    }
    h->phase(7, 5);
    pm_fft_r2c_x(l2, noise, h->Np(), h->spec, SS, nslots, h->d_tw[l2], st);
    pm_fft_y(l2, h->spec, SS, nslots, -1, h->d_tw[l2], st);
    PmZPass z{};
    z.in[0] = h->spec;
    for (int c = 0; c < 3; ++c) z.out[c] = h->spec + c * S;
    z.slot_stride = SS;
    z.tw = h->d_tw[l2];
    z.ictab = h->d_ictab;
    z.kf = (float)(2.0 * M_PI / h->cfg.box);
    pm_fft_z(l2, PM_Z_IC, z, nslots, st);
    pm_fft_y(l2, h->spec, S, 3 * nslots, 1, h->d_tw[l2], st);
    const float Dini = (float)h->growth->D(h->cfg.a_ini);
    pm_fft_c2r_x(l2, h->spec, S, vel, h->Np(), disp, h->Np(), Dini, 3 * nslots, h->d_tw[l2], st);
    h->phase_end();
    return h->check_launch("zeldovich ic");
}

}  // namespace

extern "C" {

void pm_config_default(pm_config* c) {
    if (!c) return;
    std::memset(c, 0, sizeof *c);
    c->n_part = 64;
    c->n_mesh = 64;
    c->box = 256.0;
    c->order = 2;
    c->interlace = 0;
    c->grad_order = 4;
    c->lap_order = 0;
    c->omega_m = 0.3;
    c->h = 0.7;
    c->n_s = 0.96;
    c->sigma8 = 0.8;
    c->a_ini = 0.02;
    c->a_end = 1.0;
    c->n_steps = 6;
    c->stepper = 0;
    c->time_var = 0;
    c->zero_corner = 1;
    c->batch = 1;
    c->pk_mesh_max = 0;
    c->deconvolve = 0;
    c->lpt_order = 1;
}

int pm_workspace_bytes(const pm_config* cfg, size_t* bytes) {
    std::string why;
    int rc = validate(cfg, why);
    if (rc) { g_init_error = why; return rc; }
    if (!bytes) { g_init_error = "bytes is NULL"; return PM_ERR_ARG; }
    *bytes = workspace_bytes(cfg);
    return PM_OK;
}

int pm_init(const pm_config* cfg, void* stream, pm_handle** out) {
    if (!out) { g_init_error = "out is NULL"; return PM_ERR_ARG; }
    *out = nullptr;
    std::string why;
    int rc = validate(cfg, why);
    if (rc) { g_init_error = why; return rc; }
    auto h = std::make_unique<pm_handle>();
    h->cfg = *cfg;
    h->stream = (cudaStream_t)stream;
    h->B = cfg->batch;
    h->np = cfg->n_part;
    h->ng = cfg->nufft ? 2 * cfg->n_mesh : cfg->n_mesh;   // NUFFT: meshes on the upsampled grid
    h->mak = cfg->nufft ? 5 : cfg->order;
    h->npk = cfg->pk_mesh_max ? cfg->pk_mesh_max : cfg->n_mesh;
    h->nmax = std::max(h->ng, std::max(h->np, h->npk));
    h->ngrids = cfg->interlace ? 2 : 1;
    h->ncomp = cfg->interlace ? 6 : 3;
    // host tables (App. B, Sec. 2.4)
    h->growth = std::make_unique<pmcosmo::Growth>(cfg->omega_m);
    h->table = pmcosmo::step_table(*h->growth, cfg->a_ini, cfg->a_end, cfg->n_steps, cfg->stepper, cfg->time_var);
    h->tables_by_nsteps[cfg->n_steps] = h->table;

    auto bail = [&](int code) {
        g_init_error = h->err;
        pm_destroy(h.release());
        return code;
    };
    const int B = h->B;
    if ((rc = dalloc(h.get(), &h->rho, (size_t)B * h->rho_slot(), "density"))) return bail(rc);
    if ((rc = dalloc(h.get(), &h->spec, (size_t)B * h->spec_slot(), "spectra"))) return bail(rc);
    const long long f4 = std::max((long long)h->ngrids * h->Mg(), cfg->lpt_order == 2 ? (long long)h->Np() : 0ll);
    if ((rc = dalloc(h.get(), &h->force, (size_t)B * f4, "force meshes"))) return bail(rc);
    if ((rc = dalloc(h.get(), &h->d_table, (size_t)cfg->n_steps, "step table"))) return bail(rc);
    if ((rc = dalloc(h.get(), &h->d_slots, (size_t)B, "slot table"))) return bail(rc);
    if ((rc = dalloc(h.get(), &h->d_unit, 1, "unit coef"))) return bail(rc);
    // twiddles for every size a call may use (P(k) and density meshes may be smaller than n_mesh)
    for (int n = 16; n <= h->nmax; n *= 2)
        if ((rc = upload_twiddles(h.get(), n))) return bail(rc);
    // the padding columns of the spectra are transformed by the column passes: keep them finite
    if (cudaMemset(h->spec, 0, sizeof(float2) * B * h->spec_slot()) != cudaSuccess) {
        h->fail(PM_ERR_CUDA, "memset spectra");
        return bail(PM_ERR_CUDA);
    }
    {
        std::vector<SlotCoef> t(cfg->n_steps);
        for (int i = 0; i < cfg->n_steps; ++i) t[i] = to_slot(h->table[i]);
        SlotCoef unit{};
        unit.active = 1;
        std::vector<SlotCoef> idle(B);
        if (cudaMemcpy(h->d_table, t.data(), t.size() * sizeof(SlotCoef), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->d_unit, &unit, sizeof unit, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(h->d_slots, idle.data(), B * sizeof(SlotCoef), cudaMemcpyHostToDevice) != cudaSuccess) {
            h->fail(PM_ERR_CUDA, "upload coefficient tables");
            return bail(PM_ERR_CUDA);
        }
    }
    {
        // force kernels of Table 2 per DFT bin (FP64 on the host, stored FP32)
        const int n = h->ng;
        const double H = cfg->box / n;
        std::vector<float> lap(n), grad(n);
        for (int j = 0; j < n; ++j) {
            const int m = j < n / 2 ? j : j - n;
            const double k = 2.0 * M_PI * m / cfg->box;
            lap[j] = (float)lap1d(k, H, cfg->lap_order);
            grad[j] = (j == n / 2) ? 0.f : (float)grad1d(k, H, cfg->grad_order);
        }
        if ((rc = dalloc(h.get(), &h->d_lap, n, "laplacian kernel"))) return bail(rc);
        if ((rc = dalloc(h.get(), &h->d_grad, n, "gradient kernel"))) return bail(rc);
        cudaMemcpy(h->d_lap, lap.data(), n * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(h->d_grad, grad.data(), n * sizeof(float), cudaMemcpyHostToDevice);
        if (cfg->nufft) {
            // NUFFT: 1 / psi^(k)^2 per axis on the upsampled grid's bins, psi^ the continuous
            // transform of the ES kernel (width 5, beta = 11.5; Simpson in FP64), and zero
            // outside the band |m| < n_mesh / 2
            const int nb = cfg->n_mesh;
            const int q = 20000;                                  // Simpson intervals on [-2.5, 2.5]
            std::vector<double> phi(q + 1);
            for (int i = 0; i <= q; ++i) {
                const double t = -2.5 + 5.0 * i / q, z = t / 2.5, r = 1.0 - z * z;
                phi[i] = r > 0 ? std::exp(11.5 * (std::sqrt(r) - 1.0)) : (r == 0 ? std::exp(-11.5) : 0.0);
            }
            std::vector<float> dec(n);
            for (int j = 0; j < n; ++j) {
                const int m = j < n / 2 ? j : j - n;
                if (std::abs(m) >= nb / 2) {
                    dec[j] = 0.f;
                    continue;
                }
                const double kap = 2.0 * M_PI * m / n;
                double sum = 0;
                for (int i = 0; i <= q; ++i) {
                    const double t = -2.5 + 5.0 * i / q;
                    const double wgt = (i == 0 || i == q) ? 1.0 : (i % 2 ? 4.0 : 2.0);
                    sum += wgt * phi[i] * std::cos(kap * t);
                }
                const double ph = sum * (5.0 / q) / 3.0;
                dec[j] = (float)(1.0 / (ph * ph));
            }
            if ((rc = dalloc(h.get(), &h->d_dec, n, "nufft deconvolution"))) return bail(rc);
            cudaMemcpy(h->d_dec, dec.data(), n * sizeof(float), cudaMemcpyHostToDevice);
        } else if (cfg->deconvolve) {
            // Table 1: W^ = sinc^p(kt/2), sinc(x) = sin(pi x)/(pi x), kt = k/k_Ny = 2 m / n;
            // the deposit and the interpolation each apply it once: divide by W^2
            std::vector<float> dec(n);
            for (int j = 0; j < n; ++j) {
                const int m = j < n / 2 ? j : j - n;
                const double x = M_PI * m / n;                 // pi kt / 2
                const double s = m == 0 ? 1.0 : std::sin(x) / x;
                dec[j] = (float)std::pow(s, -2.0 * cfg->order);
            }
            if ((rc = dalloc(h.get(), &h->d_dec, n, "deconvolution kernel"))) return bail(rc);
            cudaMemcpy(h->d_dec, dec.data(), n * sizeof(float), cudaMemcpyHostToDevice);
        }
    }
    {
        // Zel'dovich multiplier per integer |m|^2 = s (k = 2 pi sqrt(s) / L):
        // sqrt(P(k) N / L^3) / (D(1) k^2) / N, zero for s = 0 and (zero_corner) |k| > k_Ny
        const int n = h->np;
        const int ns = 3 * (n / 2) * (n / 2) + 1;
        pmcosmo::LinearSpectrum pk(cfg->omega_m, cfg->h, cfg->n_s, cfg->sigma8);
        const double D1 = h->growth->D(1.0);
        const double Np = (double)n * n * n, L3 = cfg->box * cfg->box * cfg->box;
        std::vector<float> t(ns);
        for (int s = 0; s < ns; ++s) {
            const double k = 2.0 * M_PI * std::sqrt((double)s) / cfg->box;
            const bool keep = s > 0 && (!cfg->zero_corner || s <= (n / 2) * (n / 2));
            t[s] = keep ? (float)(std::sqrt(pk(k) * Np / L3) / (D1 * k * k) / Np) : 0.f;
        }
        if ((rc = dalloc(h.get(), &h->d_ictab, ns, "IC table"))) return bail(rc);
        cudaMemcpy(h->d_ictab, t.data(), ns * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (cudaMallocHost((void**)&h->h_slots, 4 * B * sizeof(SlotCoef)) != cudaSuccess) {
        h->fail(PM_ERR_OOM, "pinned slot buffer");
        return bail(PM_ERR_OOM);
    }
    for (int i = 0; i < 4; ++i) cudaEventCreateWithFlags(&h->slot_ev[i], cudaEventDisableTiming);
    if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        h->fail(PM_ERR_CUDA, "init: %s", cudaGetErrorString(cudaGetLastError()));
        return bail(PM_ERR_CUDA);
    }
    *out = h.release();
    return PM_OK;
}

void pm_destroy(pm_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaDeviceSynchronize();
    cudaFree(h->rho);
    cudaFree(h->spec);
    cudaFree(h->force);
    cudaFree(h->d_table);
    cudaFree(h->d_slots);
    cudaFree(h->d_unit);
    for (auto* p : h->d_tw) cudaFree(p);
    cudaFree(h->d_lap);
    cudaFree(h->d_grad);
    cudaFree(h->d_dec);
    cudaFree(h->d_ictab);
    cudaFree(h->d_pk);
    cudaFree(h->adj3);
    cudaFree(h->jrho);
    cudaFree(h->jforce);
    cudaFree(h->d_dot);
    cudaFree(h->d_noise);
    cudaFree(h->d_disp);
    cudaFree(h->d_vel);
    if (h->h_slots) cudaFreeHost(h->h_slots);
    for (auto& e : h->slot_ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : h->ev_pool) cudaEventDestroy(e);
    delete h;
}

const char* pm_last_error(const pm_handle* h) { return h ? h->err.c_str() : g_init_error.c_str(); }

int pm_set_stream(pm_handle* h, void* stream) {
    if (!h) return PM_ERR_ARG;
    h->stream = (cudaStream_t)stream;
    return PM_OK;
}

int pm_step_table(const pm_handle* h, double* out, int32_t cap) {
    if (!h || !out) return PM_ERR_ARG;
    if (cap < (int)h->table.size()) return PM_ERR_ARG;
    for (size_t i = 0; i < h->table.size(); ++i) {
        const auto& c = h->table[i];
        const double row[7] = {c.tau1, c.tau2, c.alpha, c.beta, c.D_half, c.D_n, c.D_next};
        std::memcpy(out + 7 * i, row, sizeof row);
    }
    return PM_OK;
}

int pm_host_step_table(const pm_config* cfg, double* out, int32_t cap) {
    std::string why;
    int rc = validate(cfg, why);
    if (rc) { g_init_error = why; return rc; }
    if (!out || cap < cfg->n_steps) { g_init_error = "pm_host_step_table: out too small"; return PM_ERR_ARG; }
    pmcosmo::Growth g(cfg->omega_m);
    auto t = pmcosmo::step_table(g, cfg->a_ini, cfg->a_end, cfg->n_steps, cfg->stepper, cfg->time_var);
    for (size_t i = 0; i < t.size(); ++i) {
        const auto& c = t[i];
        const double row[7] = {c.tau1, c.tau2, c.alpha, c.beta, c.D_half, c.D_n, c.D_next};
        std::memcpy(out + 7 * i, row, sizeof row);
    }
    return PM_OK;
}

int pm_growth(const pm_handle* h, double a, double* out) {
    if (!h || !out || !(a > 1e-5 && a < 4.0)) return PM_ERR_ARG;
    out[0] = h->growth->D(a);
    out[1] = h->growth->E(a);
    out[2] = h->growth->dE_dD(a);
    return PM_OK;
}

int pm_ic_zeldovich(pm_handle* h, const float* noise, float* disp, float* vel) {
    if (!h) return PM_ERR_ARG;
    if (!noise || !disp || !vel) return h->fail(PM_ERR_ARG, "pm_ic_zeldovich: NULL buffer");
    return ic_impl(h, noise, disp, vel, h->B);
}

int pm_ic_zeldovich_slot(pm_handle* h, int32_t slot, const float* noise, float* disp, float* vel) {
    if (!h) return PM_ERR_ARG;
    if (!noise || !disp || !vel) return h->fail(PM_ERR_ARG, "pm_ic_zeldovich_slot: NULL buffer");
    if (slot < 0 || slot >= h->B) return h->fail(PM_ERR_ARG, "slot %d out of range [0, %d)", slot, h->B);
    return ic_impl(h, noise, disp, vel, 1);
}

int pm_step(pm_handle* h, float* disp, float* vel, int32_t step) {
    if (!h) return PM_ERR_ARG;
    if (!disp || !vel) return h->fail(PM_ERR_ARG, "pm_step: NULL buffer");
    if (step < 0 || step >= (int)h->table.size())
        return h->fail(PM_ERR_ARG, "step %d out of range [0, %d)", step, (int)h->table.size());
    return one_step(h, disp, vel, h->d_table + step, 0);
}

int pm_run(pm_handle* h, float* disp, float* vel, int32_t b, int32_t e) {
    if (!h) return PM_ERR_ARG;
    if (!disp || !vel) return h->fail(PM_ERR_ARG, "pm_run: NULL buffer");
    if (b < 0 || e < b || e > (int)h->table.size())
        return h->fail(PM_ERR_ARG, "pm_run: bad step range [%d, %d)", b, e);
    if (e == b) return PM_OK;
    // Between the steps of a run the positions are carried already drifted by
    // the next step's tau1 (X_half - q), so each later deposit reads positions only.
    const bool predrift = h->ngrids == 1 && e - b >= 2;
    if (!predrift) {
        for (int s = b; s < e; ++s) {
            int rc = pm_step(h, disp, vel, s);
            if (rc) return rc;
        }
        return PM_OK;
    }
    cudaStream_t st = h->stream;
    const long long Mg = h->Mg();
    const PmGeom gd = geom(h, h->ng, h->rho_slot());
    const PmGeom gf = geom(h, h->ng, Mg);
    for (int s = b; s < e; ++s) {
        // later steps find the density zeroed by the previous step's forward x pass
        if (s == b && cudaMemsetAsync(h->rho, 0, sizeof(float) * h->rho_slot() * h->B, st) != cudaSuccess)
            return h->fail(PM_ERR_CUDA, "memset density");
        h->phase(0, 1);
        if (s == b)
            pm_deposit(h->mak, gd, disp, vel, h->d_table + s, 0, 0.f, h->rho, h->B, st);
        else
            pm_deposit(h->mak, gd, disp, nullptr, h->d_unit, 0, 0.f, h->rho, h->B, st);
        h->phase_end();
        int rc = spectral_force(h, h->rho, h->rho_slot(), Mg, (float)(1.0 / (double)h->Np()), nullptr, h->force, h->B,
                                s + 1 < e);
        if (rc) return rc;
        h->phase(6, 1);
        pm_interp_kick(h->mak, 0, gf, disp, vel, h->d_table + s, 0, h->force, h->B, st, s > b,
                       s + 1 < e ? h->d_table + s + 1 : nullptr);
        h->phase_end();
        if ((rc = h->check_launch("pm_run step"))) return rc;
    }
    return PM_OK;
}

int pm_set_slots(pm_handle* h, const int32_t* n_steps, const int32_t* step) {
    if (!h) return PM_ERR_ARG;
    if (!n_steps || !step) return h->fail(PM_ERR_ARG, "pm_set_slots: NULL array");
    const int r = h->slot_ring;
    h->slot_ring = (r + 1) % 4;
    // the pinned buffer of this ring entry may still feed an earlier copy
    cudaEventSynchronize(h->slot_ev[r]);
    SlotCoef* hs = h->h_slots + (size_t)r * h->B;
    for (int s = 0; s < h->B; ++s) {
        SlotCoef c{};
        if (step[s] >= 0) {
            const int ns = n_steps[s];
            if (ns < 1 || ns > 100000 || step[s] >= ns)
                return h->fail(PM_ERR_ARG, "slot %d: step %d of %d out of range", s, step[s], ns);
            auto it = h->tables_by_nsteps.find(ns);
            if (it == h->tables_by_nsteps.end())
                it = h->tables_by_nsteps.emplace(ns, pmcosmo::step_table(*h->growth, h->cfg.a_ini, h->cfg.a_end, ns,
                                                                        h->cfg.stepper, h->cfg.time_var)).first;
            c = to_slot(it->second[step[s]]);
        }
        hs[s] = c;
    }
    if (cudaMemcpyAsync(h->d_slots, hs, h->B * sizeof(SlotCoef), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return h->fail(PM_ERR_CUDA, "pm_set_slots: copy");
    cudaEventRecord(h->slot_ev[r], h->stream);
    return PM_OK;
}

int pm_step_slots(pm_handle* h, float* disp, float* vel) {
    if (!h) return PM_ERR_ARG;
    if (!disp || !vel) return h->fail(PM_ERR_ARG, "pm_step_slots: NULL buffer");
    return one_step(h, disp, vel, h->d_slots, 1);
}

namespace {
int pk_check(pm_handle* h, int32_t n, int32_t nbins) {
    if (!pow2_in_range(n) || n > h->npk)
        return h->fail(PM_ERR_ARG, "P(k) mesh %d must be a power of two in [16, %d]", n, h->npk);
    if (nbins < 1 || nbins > n) return h->fail(PM_ERR_ARG, "n_bins must be in [1, %d]", n);
    return PM_OK;
}

// deposit, forward transform and binning of every slot; the FP64 sums over each
// bin of w |rho^|^2 land in sums [slot][nbins] (device), asynchronously
int pk_enqueue(pm_handle* h, const float* disp, int32_t n, int32_t nbins, double* sums) {
    int rc;
    const pm_handle::BinTable* bt = nullptr;
    if ((rc = bintab_for(h, n, nbins, &bt))) return rc;
    cudaStream_t st = h->stream;
    const int l2 = ilog2i(n);
    cudaMemsetAsync(h->rho, 0, sizeof(float) * h->rho_slot() * h->B, st);
    cudaMemsetAsync(sums, 0, sizeof(double) * h->B * nbins, st);
    h->phase(8, 4);
    pm_deposit(2, geom(h, n, h->rho_slot()), disp, nullptr, h->d_unit, 0, 0.f, h->rho, h->B, st);
    pm_fft_r2c_x(l2, h->rho, h->rho_slot(), h->spec, h->spec_slot(), h->B, h->d_tw[l2], st);
    pm_fft_y(l2, h->spec, h->spec_slot(), h->B, -1, h->d_tw[l2], st);
    PmZPass z{};
    z.in[0] = h->spec;
    z.slot_stride = h->spec_slot();
    z.tw = h->d_tw[l2];
    z.pk_out = sums;
    z.nbins = nbins;
    pm_fft_z(l2, PM_Z_PK, z, h->B, st);
    h->phase_end();
    return h->check_launch("power spectrum");
}

// k, P(k) and mode counts from the bin sums (host arithmetic only)
int pk_finish(pm_handle* h, int32_t n, int32_t nbins, const double* acc, double* k, double* pk, int64_t* nmodes) {
    int rc;
    const pm_handle::BinTable* bt = nullptr;
    if ((rc = bintab_for(h, n, nbins, &bt))) return rc;
    const long long M = mesh_elems(n);
    const double L = h->cfg.box, kf = 2.0 * M_PI / L;
    const double MN = (double)M / (double)h->Np();            // delta^ = (M/N) rho^ for k != 0
    for (int b = 0; b < h->B; ++b) {
        for (int i = 0; i < nbins; ++i) {
            const double cnt = bt->count[i];
            const size_t o = (size_t)b * nbins + i;
            nmodes[o] = (int64_t)std::llround(cnt);
            k[o] = cnt > 0 ? bt->ksum[i] / cnt * kf : 0.0;
            pk[o] = cnt > 0 ? acc[o] / cnt * MN * MN * L * L * L / ((double)M * (double)M) : 0.0;
        }
    }
    return PM_OK;
}
}  // namespace

int pm_power_spectrum(pm_handle* h, const float* disp, int32_t n, int32_t nbins, double* k, double* pk,
                      int64_t* nmodes) {
    if (!h) return PM_ERR_ARG;
    if (!disp || !k || !pk || !nmodes) return h->fail(PM_ERR_ARG, "pm_power_spectrum: NULL buffer");
    int rc;
    if ((rc = pk_check(h, n, nbins))) return rc;
    if (nbins > h->pk_bins_cap) {
        cudaFree(h->d_pk);
        h->d_pk = nullptr;
        if ((rc = dalloc(h, &h->d_pk, (size_t)h->B * nbins, "P(k) bins"))) return rc;
        h->pk_bins_cap = nbins;
    }
    if ((rc = pk_enqueue(h, disp, n, nbins, h->d_pk))) return rc;
    std::vector<double> acc((size_t)h->B * nbins);
    cudaStream_t st = h->stream;
    if (cudaMemcpyAsync(acc.data(), h->d_pk, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return h->fail(PM_ERR_CUDA, "power spectrum readback: %s", cudaGetErrorString(cudaGetLastError()));
    return pk_finish(h, n, nbins, acc.data(), k, pk, nmodes);
}

int pm_power_spectrum_async(pm_handle* h, const float* disp, int32_t n_mesh, int32_t n_bins, double* bin_sums) {
    if (!h) return PM_ERR_ARG;
    if (!disp || !bin_sums) return h->fail(PM_ERR_ARG, "pm_power_spectrum_async: NULL buffer");
    int rc;
    if ((rc = pk_check(h, n_mesh, n_bins))) return rc;
    return pk_enqueue(h, disp, n_mesh, n_bins, bin_sums);
}

int pm_power_spectrum_finish(pm_handle* h, int32_t n_mesh, int32_t n_bins, const double* bin_sums, double* k,
                             double* pk, int64_t* n_modes) {
    if (!h) return PM_ERR_ARG;
    if (!bin_sums || !k || !pk || !n_modes) return h->fail(PM_ERR_ARG, "pm_power_spectrum_finish: NULL buffer");
    int rc;
    if ((rc = pk_check(h, n_mesh, n_bins))) return rc;
    return pk_finish(h, n_mesh, n_bins, bin_sums, k, pk, n_modes);
}

namespace {
int jvp_alloc(pm_handle* h);   // tangent density and force mesh, allocated on first use
}

int pm_power_spectrum_jvp(pm_handle* h, const float* disp, const float* tdisp, int32_t n, int32_t nbins, double* k,
                          double* pk, double* dpk, int64_t* nmodes) {
    if (!h) return PM_ERR_ARG;
    if (!tdisp || !dpk) return h->fail(PM_ERR_ARG, "pm_power_spectrum_jvp: NULL buffer");
    // P(k) itself (allocates and validates as pm_power_spectrum)
    int rc = pm_power_spectrum(h, disp, n, nbins, k, pk, nmodes);
    if (rc) return rc;
    if ((rc = jvp_alloc(h))) return rc;
    const pm_handle::BinTable* bt = nullptr;
    if ((rc = bintab_for(h, n, nbins, &bt))) return rc;
    cudaStream_t st = h->stream;
    const int l2 = ilog2i(n);
    const long long S = spec_elems(n);
    // the CIC density of X and its tangent along X' on the n-mesh; then the binned
    // cross spectrum 2 Re(conj(delta^) delta'^) (rho tangent in the second spectrum)
    cudaMemsetAsync(h->rho, 0, sizeof(float) * h->rho_slot() * h->B, st);
    cudaMemsetAsync(h->jrho, 0, sizeof(float) * h->rho_slot() * h->B, st);
    cudaMemsetAsync(h->d_pk, 0, sizeof(double) * h->B * nbins, st);
    pm_jvp_drift_deposit(2, 0, geom(h, n, h->rho_slot()), const_cast<float*>(disp), nullptr,
                         const_cast<float*>(tdisp), nullptr, h->d_unit, 0, h->rho, h->jrho, h->B, st);
    pm_fft_r2c_x(l2, h->rho, h->rho_slot(), h->spec, h->spec_slot(), h->B, h->d_tw[l2], st);
    pm_fft_r2c_x(l2, h->jrho, h->rho_slot(), h->spec + S, h->spec_slot(), h->B, h->d_tw[l2], st);
    pm_fft_y(l2, h->spec, h->spec_slot(), h->B, -1, h->d_tw[l2], st);
    pm_fft_y(l2, h->spec + S, h->spec_slot(), h->B, -1, h->d_tw[l2], st);
    PmZPass z{};
    z.in[0] = h->spec;
    z.in[1] = h->spec + S;
    z.slot_stride = h->spec_slot();
    z.tw = h->d_tw[l2];
    z.pk_out = h->d_pk;
    z.nbins = nbins;
    pm_fft_z(l2, PM_Z_PKX, z, h->B, st);
    if ((rc = h->check_launch("power spectrum jvp"))) return rc;
    std::vector<double> acc((size_t)h->B * nbins);
    if (cudaMemcpyAsync(acc.data(), h->d_pk, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return h->fail(PM_ERR_CUDA, "power spectrum jvp readback: %s", cudaGetErrorString(cudaGetLastError()));
    const long long M = mesh_elems(n);
    const double L = h->cfg.box, MN = (double)M / (double)h->Np();
    for (int b = 0; b < h->B; ++b)
        for (int i = 0; i < nbins; ++i) {
            const double cnt = bt->count[i];
            const size_t o = (size_t)b * nbins + i;
            dpk[o] = cnt > 0 ? acc[o] / cnt * MN * MN * L * L * L / ((double)M * (double)M) : 0.0;
        }
    return PM_OK;
}

int pm_density(pm_handle* h, const float* disp, int32_t n, int32_t order, float* delta) {
    if (!h) return PM_ERR_ARG;
    if (!disp || !delta) return h->fail(PM_ERR_ARG, "pm_density: NULL buffer");
    if (!pow2_in_range(n)) return h->fail(PM_ERR_ARG, "mesh %d must be a power of two in [16, 1024]", n);
    if (order < 2 || order > 4) return h->fail(PM_ERR_ARG, "order must be 2, 3 or 4");
    const long long M = mesh_elems(n);
    cudaStream_t st = h->stream;
    cudaMemsetAsync(delta, 0, sizeof(float) * M * h->B, st);
    pm_deposit(order, geom(h, n, M), disp, nullptr, h->d_unit, 0, 0.f, delta, h->B, st);
    const long long tot = M * h->B;
    k_affine<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(delta, tot, (float)((double)M / (double)h->Np()), -1.f);
    return h->check_launch("pm_density");
}

int pm_force_mesh(pm_handle* h, const float* delta, float* force) {
    if (h && h->cfg.nufft) return h->fail(PM_ERR_UNSUPPORTED, "pm_force_mesh: not available with the NUFFT force");
    if (!h) return PM_ERR_ARG;
    if (!delta || !force) return h->fail(PM_ERR_ARG, "pm_force_mesh: NULL buffer");
    if (h->ngrids != 1) return h->fail(PM_ERR_UNSUPPORTED, "pm_force_mesh: single grid only");
    return spectral_force(h, delta, h->Mg(), 0, (float)(1.0 / (double)h->Mg()), force, nullptr, h->B);
}

int pm_interp(pm_handle* h, const float* disp, const float* force, float* acc) {
    if (h && h->cfg.nufft) return h->fail(PM_ERR_UNSUPPORTED, "pm_interp: not available with the NUFFT force");
    if (!h) return PM_ERR_ARG;
    if (!disp || !force || !acc) return h->fail(PM_ERR_ARG, "pm_interp: NULL buffer");
    if (h->ngrids != 1) return h->fail(PM_ERR_UNSUPPORTED, "pm_interp: single grid only");
    pm_interp(h->cfg.order, 0, geom(h, h->ng, 3 * h->Mg()), disp, force, acc, h->B, h->stream);
    return h->check_launch("pm_interp");
}

namespace {
int jvp_alloc(pm_handle* h) {
    if (h->jrho) return PM_OK;
    int rc = dalloc(h, &h->jrho, (size_t)h->B * h->rho_slot(), "tangent density");
    if (rc) return rc;
    return dalloc(h, &h->jforce, (size_t)h->B * h->Mg(), "tangent force mesh");
}

int adj_alloc(pm_handle* h) {
    if (h->adj3) return PM_OK;
    int rc = dalloc(h, &h->adj3, (size_t)h->B * 3 * std::max(h->Mg(), h->Np()), "adjoint meshes");
    if (rc) return rc;
    return dalloc(h, &h->d_dot, (size_t)h->B, "adjoint dot");
}
}  // namespace

int pm_jvp(pm_handle* h, float* disp, float* vel, float* tdisp, float* tvel, int32_t b, int32_t e) {
    if (h && h->cfg.nufft) return h->fail(PM_ERR_UNSUPPORTED, "pm_jvp: not available with the NUFFT force");
    if (!h) return PM_ERR_ARG;
    if (!disp || !vel || !tdisp || !tvel) return h->fail(PM_ERR_ARG, "pm_jvp: NULL buffer");
    if (h->ngrids != 1) return h->fail(PM_ERR_UNSUPPORTED, "pm_jvp: interlaced grids are not supported");
    if (b < 0 || e < b || e > (int)h->table.size())
        return h->fail(PM_ERR_ARG, "pm_jvp: bad step range [%d, %d)", b, e);
    int rc;
    if ((rc = jvp_alloc(h))) return rc;
    cudaStream_t st = h->stream;
    const int n = h->ng, order = h->cfg.order;
    const long long Mg = h->Mg();
    const PmGeom gd = geom(h, n, h->rho_slot());
    const PmGeom gf = geom(h, n, Mg);
    const float scale = (float)(1.0 / (double)h->Np());
    for (int s = b; s < e; ++s) {
        const SlotCoef* coef = h->d_table + s;
        cudaMemsetAsync(h->rho, 0, sizeof(float) * h->rho_slot() * h->B, st);
        cudaMemsetAsync(h->jrho, 0, sizeof(float) * h->rho_slot() * h->B, st);
        h->phase(0, 1);
        pm_jvp_drift_deposit(order, 1, gd, disp, vel, tdisp, tvel, coef, 0, h->rho, h->jrho, h->B, st);
        h->phase_end();
        if ((rc = spectral_force(h, h->rho, h->rho_slot(), Mg, scale, nullptr, h->force, h->B))) return rc;
        if ((rc = spectral_force(h, h->jrho, h->rho_slot(), Mg, scale, nullptr, h->jforce, h->B))) return rc;
        h->phase(6, 1);
        pm_jvp_interp_kick(order, gf, disp, vel, tdisp, tvel, coef, 0, h->force, h->jforce, h->B, st);
        h->phase_end();
        if ((rc = h->check_launch("pm_jvp step"))) return rc;
    }
    return PM_OK;
}

int pm_adjoint(pm_handle* h, float* disp, float* vel, float* adisp, float* avel, int32_t step_end) {
    if (h && h->cfg.nufft) return h->fail(PM_ERR_UNSUPPORTED, "pm_adjoint: not available with the NUFFT force");
    if (!h) return PM_ERR_ARG;
    if (!disp || !vel || !adisp || !avel) return h->fail(PM_ERR_ARG, "pm_adjoint: NULL buffer");
    if (h->ngrids != 1) return h->fail(PM_ERR_UNSUPPORTED, "pm_adjoint: interlaced grids are not supported");
    if (step_end < 0 || step_end > (int)h->table.size())
        return h->fail(PM_ERR_ARG, "pm_adjoint: step_end %d out of [0, %d]", step_end, (int)h->table.size());
    int rc;
    if ((rc = adj_alloc(h))) return rc;
    cudaStream_t st = h->stream;
    const int n = h->ng, l2 = ilog2i(n), order = h->cfg.order;
    const long long Mg = h->Mg(), S = spec_elems(n);
    const PmGeom gd = geom(h, n, h->rho_slot());
    const PmGeom g3 = geom(h, n, 3 * Mg);
    for (int s = step_end - 1; s >= 0; --s) {
        const SlotCoef* coef = h->d_table + s;
        cudaMemsetAsync(h->rho, 0, sizeof(float) * h->rho_slot() * h->B, st);
        h->phase(0, 1);
        pm_adj_drift_deposit(order, gd, disp, vel, adisp, avel, coef, 0, h->rho, h->B, st);
        h->phase_end();
        if ((rc = spectral_force(h, h->rho, h->rho_slot(), Mg, (float)(1.0 / (double)h->Np()), nullptr, h->force,
                                 h->B)))
            return rc;
        cudaMemsetAsync(h->adj3, 0, sizeof(float) * 3 * Mg * h->B, st);
        h->phase(6, 1);
        pm_adj_interp(order, g3, disp, vel, adisp, avel, coef, 0, h->force, h->adj3, h->B, st);
        h->phase_end();
        // rho* = sum_c G_c^T s_c, G_c^T = (1/N) IDFT diag(conj m_c) DFT
        h->phase(9, 5);
        if (h->cfg.grad_order != 0) {
            // finite-difference gradient: G_c^T s_c summed = Lap^-1 (sum_c D1_c s_c), the divergence
            // stencil in real space and one potential solve (the z pass of the forward force)
            pm_div_stencil(h->cfg.grad_order, l2, (float)(n / h->cfg.box), h->adj3, 3 * Mg, h->rho, h->rho_slot(), h->B,
                           st);
            pm_fft_r2c_x(l2, h->rho, h->rho_slot(), h->spec, S, h->B, h->d_tw[l2], st);
            pm_fft_y(l2, h->spec, S, h->B, -1, h->d_tw[l2], st);
            PmZPass z{};
            z.in[0] = h->spec;
            z.out[0] = h->spec;
            z.slot_stride = S;
            z.tw = h->d_tw[l2];
            z.lap1 = h->d_lap;
            z.grad1 = h->d_grad;
            z.dec1 = h->d_dec;
            z.scale = (float)(1.0 / (double)h->Np());
            pm_fft_z(l2, PM_Z_POT, z, h->B, st);
            pm_fft_y(l2, h->spec, S, h->B, 1, h->d_tw[l2], st);
            pm_fft_c2r_x(l2, h->spec, S, h->rho, h->rho_slot(), nullptr, 0, 0.f, h->B, h->d_tw[l2], st);
        } else {
            pm_fft_r2c_x(l2, h->adj3, Mg, h->spec, S, 3 * h->B, h->d_tw[l2], st);
            pm_fft_y(l2, h->spec, S, 3 * h->B, -1, h->d_tw[l2], st);
            PmZPass z{};
            for (int c = 0; c < 3; ++c) z.in[c] = h->spec + c * S;
            z.out[0] = h->spec;
            z.slot_stride = 3 * S;
            z.tw = h->d_tw[l2];
            z.lap1 = h->d_lap;
            z.grad1 = h->d_grad;
            z.dec1 = h->d_dec;
            z.scale = (float)(1.0 / (double)h->Np());
            pm_fft_z(l2, PM_Z_ADJ, z, h->B, st);
            pm_fft_y(l2, h->spec, 3 * S, h->B, 1, h->d_tw[l2], st);
            pm_fft_c2r_x(l2, h->spec, 3 * S, h->rho, h->rho_slot(), nullptr, 0, 0.f, h->B, h->d_tw[l2], st);
        }
        h->phase_end();
        h->phase(6, 1);
        pm_adj_gather_grad(order, 1, gd, disp, vel, adisp, avel, coef, 0, h->rho, 0.f, h->B, st);
        h->phase_end();
        if ((rc = h->check_launch("pm_adjoint step"))) return rc;
    }
    return PM_OK;
}

int pm_ic_adjoint(pm_handle* h, const float* noise, const float* adisp, const float* avel, float* anoise,
                  double* dsigma8) {
    if (!h) return PM_ERR_ARG;
    if (!noise || !adisp || !avel || !anoise) return h->fail(PM_ERR_ARG, "pm_ic_adjoint: NULL buffer");
    if (h->cfg.lpt_order == 2)
        return h->fail(PM_ERR_UNSUPPORTED, "pm_ic_adjoint: the pullback is implemented for Zel'dovich ICs only");
    int rc;
    if ((rc = adj_alloc(h))) return rc;
    cudaStream_t st = h->stream;
    const int n = h->np, l2 = ilog2i(n);
    const long long Np = h->Np(), S = spec_elems(n);
    // psi1* = D(a_ini) X*0 + V*0  (Psi0 = D psi1, V0 = psi1)
    const float Dini = (float)h->growth->D(h->cfg.a_ini);
    pm_axpby(h->adj3, adisp, avel, Dini, 1.f, 3 * Np * h->B, st);
    // w* = sum_c F_IC,c^T psi1*_c
    pm_fft_r2c_x(l2, h->adj3, Np, h->spec, S, 3 * h->B, h->d_tw[l2], st);
    pm_fft_y(l2, h->spec, S, 3 * h->B, -1, h->d_tw[l2], st);
    PmZPass z{};
    for (int c = 0; c < 3; ++c) z.in[c] = h->spec + c * S;
    z.out[0] = h->spec;
    z.slot_stride = 3 * S;
    z.tw = h->d_tw[l2];
    z.ictab = h->d_ictab;
    z.kf = (float)(2.0 * M_PI / h->cfg.box);
    pm_fft_z(l2, PM_Z_IC_ADJ, z, h->B, st);
    pm_fft_y(l2, h->spec, 3 * S, h->B, 1, h->d_tw[l2], st);
    pm_fft_c2r_x(l2, h->spec, 3 * S, anoise, Np, nullptr, 0, 0.f, h->B, h->d_tw[l2], st);
    if ((rc = h->check_launch("pm_ic_adjoint"))) return rc;
    if (dsigma8) {
        // psi1 is linear in the noise and proportional to sigma8: dL/dsigma8 = <w*, w> / sigma8
        cudaMemsetAsync(h->d_dot, 0, sizeof(double) * h->B, st);
        pm_dot(anoise, noise, Np, h->d_dot, h->B, st);
        std::vector<double> d(h->B);
        if (cudaMemcpyAsync(d.data(), h->d_dot, sizeof(double) * h->B, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return h->fail(PM_ERR_CUDA, "pm_ic_adjoint: readback");
        for (int b = 0; b < h->B; ++b) dsigma8[b] = d[b] / h->cfg.sigma8;
    }
    return h->check_launch("pm_ic_adjoint");
}

int pm_density_vjp(pm_handle* h, const float* disp, int32_t n, int32_t order, const float* ddelta, float* adisp) {
    if (h && h->cfg.nufft) return h->fail(PM_ERR_UNSUPPORTED, "pm_density_vjp: not available with the NUFFT force");
    if (!h) return PM_ERR_ARG;
    if (!disp || !ddelta || !adisp) return h->fail(PM_ERR_ARG, "pm_density_vjp: NULL buffer");
    if (!pow2_in_range(n)) return h->fail(PM_ERR_ARG, "mesh %d must be a power of two in [16, 1024]", n);
    if (order < 2 || order > 4) return h->fail(PM_ERR_ARG, "order must be 2, 3 or 4");
    const long long M = mesh_elems(n);
    // delta = (M/N) sum_i W(r_j - X_i) - 1  =>  X*_i = (M/N) sum_j delta*_j d/dX_i W(r_j - X_i)
    pm_adj_gather_grad(order, 0, geom(h, n, M), const_cast<float*>(disp), nullptr, adisp, nullptr, nullptr, 0, ddelta,
                       (float)((double)M / (double)h->Np()), h->B, h->stream);
    return h->check_launch("pm_density_vjp");
}

int pm_profile(pm_handle* h, int32_t enable) {
    if (!h) return PM_ERR_ARG;
    h->prof = enable != 0;
    h->ev_marks.clear();
    for (auto& c : h->launches) c = 0;
    return PM_OK;
}

int pm_profile_read(pm_handle* h, double* ms, int64_t* calls, int64_t* launches, int32_t cap) {
    if (!h || !ms || !calls || !launches || cap < PM_NPHASE) return PM_ERR_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return h->fail(PM_ERR_CUDA, "pm_profile_read: sync");
    for (int p = 0; p < PM_NPHASE; ++p) { ms[p] = 0.0; calls[p] = 0; launches[p] = h->launches[p]; }
    for (auto& m : h->ev_marks) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, h->ev_pool[m.second], h->ev_pool[m.second + 1]) == cudaSuccess) {
            ms[m.first] += t;
            calls[m.first] += 1;
        }
    }
    cudaGetLastError();
    return PM_OK;
}

namespace {
// host-buffer modes: upload the noise, ICs and the whole run into the handle's
// device state buffers (allocated on first use)
int host_mode_run(pm_handle* h, const float* noise) {
    int rc;
    const size_t Nb = (size_t)h->Np() * h->B;
    if (!h->d_noise) {
        if ((rc = dalloc(h, &h->d_noise, Nb, "host-mode noise"))) return rc;
        if ((rc = dalloc(h, &h->d_disp, 3 * Nb, "host-mode disp"))) return rc;
        if ((rc = dalloc(h, &h->d_vel, 3 * Nb, "host-mode vel"))) return rc;
    }
    if (cudaMemcpyAsync(h->d_noise, noise, Nb * 4, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return h->fail(PM_ERR_CUDA, "noise upload");
    if ((rc = ic_impl(h, h->d_noise, h->d_disp, h->d_vel, h->B))) return rc;
    return pm_run(h, h->d_disp, h->d_vel, 0, (int)h->table.size());
}
}  // namespace

int pm_simulate_pk_host(pm_handle* h, const float* noise, int32_t n_mesh, int32_t n_bins, double* k, double* pk,
                        int64_t* n_modes) {
    if (!h) return PM_ERR_ARG;
    if (!noise || !k || !pk || !n_modes) return h->fail(PM_ERR_ARG, "pm_simulate_pk_host: NULL buffer");
    if (!pow2_in_range(n_mesh) || n_mesh > h->npk)
        return h->fail(PM_ERR_ARG, "P(k) mesh %d must be a power of two in [16, %d]", n_mesh, h->npk);
    if (n_bins < 1 || n_bins > n_mesh) return h->fail(PM_ERR_ARG, "n_bins must be in [1, %d]", n_mesh);
    int rc;
    if ((rc = host_mode_run(h, noise))) return rc;
    return pm_power_spectrum(h, h->d_disp, n_mesh, n_bins, k, pk, n_modes);
}

int pm_simulate_host(pm_handle* h, const float* noise, float* disp, float* vel) {
    if (!h) return PM_ERR_ARG;
    if (!noise || !disp || !vel) return h->fail(PM_ERR_ARG, "pm_simulate_host: NULL buffer");
    int rc;
    const size_t Nb = (size_t)h->Np() * h->B;
    cudaStream_t st = h->stream;
    if ((rc = host_mode_run(h, noise))) return rc;
    if (cudaMemcpyAsync(disp, h->d_disp, 3 * Nb * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(vel, h->d_vel, 3 * Nb * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return h->fail(PM_ERR_CUDA, "state download");
    if (cudaStreamSynchronize(st) != cudaSuccess)
        return h->fail(PM_ERR_CUDA, "pm_simulate_host: %s", cudaGetErrorString(cudaGetLastError()));
    return PM_OK;
}

}  // extern "C"
