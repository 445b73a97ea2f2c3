// Host FP64 cosmology used by the PM library (see cosmo_host.cpp).
#pragma once
#include <vector>

namespace pmcosmo {

struct Growth {
    explicit Growth(double omega_m);
    double D(double a) const;
    double E(double a) const;
    double dE_dD(double a) const;
    double dD_dlna(double a) const;
    double a_of_D(double D) const;
    double om;

private:
    void rhs(double lna, const double* y, double* dy) const;
    void rk4(double x, const double* y, double h, double* out) const;
    void at(double a, double* y) const;
    double lna0, dx;
    int nnode;
    std::vector<double> ys;
};

struct StepCoef {
    double tau1, tau2, alpha, beta, D_half, D_n, D_next;
};

// stepper 0 = BullFrog, 1 = FastPM; time_var 0 = uniform in D, 1 = uniform in a
std::vector<StepCoef> step_table(const Growth& g, double a_ini, double a_end, int n_steps, int stepper,
                                 int time_var);

double bbks_T(double k, double om, double h);

struct LinearSpectrum {
    LinearSpectrum(double om, double h, double ns, double sigma8);
    double operator()(double k) const;   // P_lin(k, a = 1), k in h/Mpc, P in (Mpc/h)^3
    double om, h, ns, A;
};

}  // namespace pmcosmo
