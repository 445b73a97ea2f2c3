// Host-side FP64 cosmology for the PM library: growth factors D(a), E(a)
// (App. B), the per-step DKD coefficients of BullFrog / FastPM (Sec. 2.4), and
// the BBKS linear power spectrum normalised to sigma_8 (the linear spectrum
// that feeds the Zel'dovich initial conditions).
//
// Conventions: flat LambdaCDM without radiation, (H/H0)^2 = Om a^-3 + 1 - Om;
// D ~ a and E ~ -3/7 D^2 for a -> 0 (the normalisation BullFrog uses).
#include "cosmo_host.h"

#include <cmath>

namespace pmcosmo {

namespace {
double h2(double a, double om) { return om / (a * a * a) + (1.0 - om); }
}  // namespace

// The growth equations in ln a (App. B), written for (D, dD/dlna, E, dE/dlna):
//   D'' = 3 gam D - (2 + dlnH/dlna) D',   E'' = 3 gam (E - D^2) - (2 + dlnH/dlna) E',
//   gam = Om / (2 a^3 H^2), dlnH/dlna = -3/2 Om a^-3 / H^2 (= -3 gam for flat LambdaCDM).
void Growth::rhs(double lna, const double* y, double* dy) const {
    const double a = std::exp(lna);
    const double hh = h2(a, om);
    const double gam = om / (2.0 * a * a * a * hh);
    const double fr = 2.0 - 1.5 * om / (a * a * a * hh);
    dy[0] = y[1];
    dy[1] = 3.0 * gam * y[0] - fr * y[1];
    dy[2] = y[3];
    dy[3] = 3.0 * gam * (y[2] - y[0] * y[0]) - fr * y[3];
}

void Growth::rk4(double x, const double* y, double h, double* out) const {
    double k1[4], k2[4], k3[4], k4[4], t[4];
    rhs(x, y, k1);
    for (int i = 0; i < 4; ++i) t[i] = y[i] + 0.5 * h * k1[i];
    rhs(x + 0.5 * h, t, k2);
    for (int i = 0; i < 4; ++i) t[i] = y[i] + 0.5 * h * k2[i];
    rhs(x + 0.5 * h, t, k3);
    for (int i = 0; i < 4; ++i) t[i] = y[i] + h * k3[i];
    rhs(x + h, t, k4);
    for (int i = 0; i < 4; ++i) out[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

Growth::Growth(double omega_m) : om(omega_m) {
    // start deep in matter domination on the growing modes D = a, E = -3/7 a^2
    lna0 = std::log(1e-5);
    const double lna1 = std::log(4.0);
    dx = 1.0 / 1024.0;
    const int n = (int)std::ceil((lna1 - lna0) / dx);
    ys.resize((size_t)(n + 1) * 4);
    const double a0 = std::exp(lna0);
    double y[4] = {a0, a0, -3.0 / 7.0 * a0 * a0, -6.0 / 7.0 * a0 * a0};
    for (int i = 0; i < 4; ++i) ys[i] = y[i];
    for (int s = 0; s < n; ++s) {
        double out[4];
        rk4(lna0 + s * dx, &ys[(size_t)s * 4], dx, out);
        for (int i = 0; i < 4; ++i) ys[(size_t)(s + 1) * 4 + i] = out[i];
    }
    nnode = n + 1;
}

void Growth::at(double a, double* y) const {
    const double x = std::log(a);
    int s = (int)std::floor((x - lna0) / dx);
    if (s < 0) s = 0;
    if (s > nnode - 2) s = nnode - 2;
    const double rem = x - (lna0 + s * dx);
    if (rem == 0.0) {
        for (int i = 0; i < 4; ++i) y[i] = ys[(size_t)s * 4 + i];
        return;
    }
    rk4(lna0 + s * dx, &ys[(size_t)s * 4], rem, y);
}

double Growth::D(double a) const { double y[4]; at(a, y); return y[0]; }
double Growth::E(double a) const { double y[4]; at(a, y); return y[2]; }
double Growth::dE_dD(double a) const { double y[4]; at(a, y); return y[3] / y[1]; }
double Growth::dD_dlna(double a) const { double y[4]; at(a, y); return y[1]; }

double Growth::a_of_D(double Dt) const {
    // D is increasing in a: bracket and bisect
    double lo = 1e-5, hi = 4.0;
    for (int it = 0; it < 200 && hi - lo > 1e-16 * hi; ++it) {
        const double mid = 0.5 * (lo + hi);
        (D(mid) < Dt ? lo : hi) = mid;
    }
    return 0.5 * (lo + hi);
}

std::vector<StepCoef> step_table(const Growth& g, double a_ini, double a_end, int n_steps, int stepper,
                                 int time_var) {
    std::vector<double> an(n_steps + 1), Dn(n_steps + 1), Dh(n_steps);
    if (time_var == 0) {              // uniform in D, midpoint centred in D
        const double D0 = g.D(a_ini), D1 = g.D(a_end), dD = (D1 - D0) / n_steps;
        for (int i = 0; i <= n_steps; ++i) Dn[i] = D0 + i * dD;
        for (int i = 0; i < n_steps; ++i) Dh[i] = D0 + (i + 0.5) * dD;
        for (int i = 0; i <= n_steps; ++i) an[i] = g.a_of_D(Dn[i]);
        an[0] = a_ini;
        an[n_steps] = a_end;
    } else {                          // uniform in a, midpoint centred in a
        const double da = (a_end - a_ini) / n_steps;
        for (int i = 0; i <= n_steps; ++i) an[i] = a_ini + i * da;
        an[n_steps] = a_end;
        for (int i = 0; i <= n_steps; ++i) Dn[i] = g.D(an[i]);
        for (int i = 0; i < n_steps; ++i) Dh[i] = g.D(a_ini + (i + 0.5) * da);
    }
    std::vector<StepCoef> out(n_steps);
    for (int i = 0; i < n_steps; ++i) {
        StepCoef c;
        c.tau1 = Dh[i] - Dn[i];
        c.tau2 = Dn[i + 1] - Dh[i];
        c.D_half = Dh[i];
        c.D_n = Dn[i];
        c.D_next = Dn[i + 1];
        if (stepper == 0) {
            // BullFrog: alpha = (E'(D_{n+1}) - xi) / (E'(D_n) - xi),
            // xi = (E_n + E'(D_n) tau1) / D_half - D_half (E' = dE/dD)
            const double En = g.E(an[i]);
            const double Ep0 = g.dE_dD(an[i]);
            const double Ep1 = g.dE_dD(an[i + 1]);
            const double xi = (En + Ep0 * c.tau1) / Dh[i] - Dh[i];
            c.alpha = (Ep1 - xi) / (Ep0 - xi);
        } else {
            // FastPM: alpha = zeta(a_n) / zeta(a_{n+1}), zeta = H a^3 dD/da = H a^2 dD/dlna
            auto zeta = [&](double a) { return std::sqrt(h2(a, g.om)) * a * a * g.dD_dlna(a); };
            c.alpha = zeta(an[i]) / zeta(an[i + 1]);
        }
        c.beta = (1.0 - c.alpha) * Dh[i];
        out[i] = c;
    }
    return out;
}

// ------------------------------------------------------------ linear spectrum
double bbks_T(double k, double om, double h) {
    const double q = k / (om * h);
    if (q <= 0.0) return 1.0;
    const double p = 1.0 + 3.89 * q + std::pow(16.1 * q, 2) + std::pow(5.46 * q, 3) + std::pow(6.71 * q, 4);
    return std::log1p(2.34 * q) / (2.34 * q) * std::pow(p, -0.25);
}

static double tophat(double x) {
    if (x < 1e-4) return 1.0 - x * x / 10.0;
    return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}

LinearSpectrum::LinearSpectrum(double om_, double h_, double ns_, double s8) : om(om_), h(h_), ns(ns_), A(1.0) {
    // sigma_8^2 = int dlnk k^3 P(k) W(8 k)^2 / (2 pi^2), composite Simpson in ln k
    const double lo = std::log(1e-6), hi = std::log(1e3);
    const int n = 1 << 19;
    const double dl = (hi - lo) / n;
    double s = 0.0;
    for (int i = 0; i <= n; ++i) {
        const double k = std::exp(lo + i * dl);
        const double w = tophat(8.0 * k);
        const double f = k * k * k * (*this)(k) * w * w;
        s += f * (i == 0 || i == n ? 1.0 : (i % 2 ? 4.0 : 2.0));
    }
    const double sig2 = s * dl / 3.0 / (2.0 * M_PI * M_PI);
    A = s8 * s8 / sig2;
}

double LinearSpectrum::operator()(double k) const {
    if (k <= 0.0) return 0.0;
    const double t = bbks_T(k, om, h);
    return A * std::pow(k, ns) * t * t;
}

}  // namespace pmcosmo
