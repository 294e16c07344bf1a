// Host cosmology for the CUDA path (float64): linear growth of a flat
// matter + Lambda universe (Sec. 3 parameters) and the BBKS linear spectrum
// normalised to sigma_8. Quadratures are composite Gauss-Legendre rules on
// fixed panels (no adaptive library routine), accurate to ~1e-13 relative.
#include <cmath>

#include "common.cuh"

namespace pmr {
namespace {

// 10-point Gauss-Legendre nodes and weights on [-1, 1] (standard table).
const double GL_X[5] = {0.1488743389816312, 0.4333953941292472, 0.6794095682990244, 0.8650633666889845,
                        0.9739065285171717};
const double GL_W[5] = {0.2955242247147529, 0.2692667193099963, 0.2190863625159820, 0.1494513491505806,
                        0.0666713443086881};

template <class F>
double gauss_legendre(F f, double a, double b, int panels) {
    double h = (b - a) / panels, sum = 0.0;
    for (int p = 0; p < panels; ++p) {
        double mid = a + (p + 0.5) * h, half = 0.5 * h;
        for (int i = 0; i < 5; ++i) sum += GL_W[i] * half * (f(mid - half * GL_X[i]) + f(mid + half * GL_X[i]));
    }
    return sum;
}

double hubble(double a, double om) { return std::sqrt(om / (a * a * a) + (1.0 - om)); }

// int_0^a da' / (a' E(a'))^3; substitute a' = t^2 so the integrand is smooth at 0:
// (a' E)^-3 = a'^{3/2} / (om + (1-om) a'^3)^{3/2}, da' = 2 t dt.
double growth_integral(double a, double om) {
    auto f = [om](double t) {
        double ap = t * t;
        double den = om + (1.0 - om) * ap * ap * ap;
        return 2.0 * t * ap * std::sqrt(ap) / (den * std::sqrt(den));
    };
    return gauss_legendre(f, 0.0, std::sqrt(a), 64);
}

double norm1(double om) { return hubble(1.0, om) * growth_integral(1.0, om); }

}  // namespace

double growth_D(double a, double om) { return hubble(a, om) * growth_integral(a, om) / norm1(om); }

double growth_dDda(double a, double om) {
    double e = hubble(a, om);
    double dE = -1.5 * om / (a * a * a * a) / e;
    double ae = a * e;
    return (dE * growth_integral(a, om) + e / (ae * ae * ae)) / norm1(om);
}

double growth_Gp(double a, double om) { return a * a * a * hubble(a, om) * growth_dDda(a, om); }

double growth_Gf(double a, double om) { return 1.5 * om * growth_D(a, om); }

double bbks_transfer(double k, double gamma) {
    if (k <= 0.0) return 1.0;
    double q = k / gamma;
    double poly = 1.0 + 3.89 * q + std::pow(16.1 * q, 2) + std::pow(5.46 * q, 3) + std::pow(6.71 * q, 4);
    return std::log(1.0 + 2.34 * q) / (2.34 * q) * std::pow(poly, -0.25);
}

double bbks_power(double k, double amp, double gamma) {
    double t = bbks_transfer(k, gamma);
    return amp * k * t * t;
}

// sigma^2(8 Mpc/h) of P = k T^2, integrated in ln k over [1e-6, 1e3] h/Mpc.
double bbks_amplitude(double sigma8, double gamma) {
    auto f = [gamma](double lnk) {
        double k = std::exp(lnk), x = 8.0 * k;
        double w = (x < 1e-3) ? 1.0 - x * x / 10.0 : 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
        return k * k * k * bbks_power(k, 1.0, gamma) * w * w;
    };
    double s2 = gauss_legendre(f, std::log(1e-6), std::log(1e3), 4000) / (2.0 * M_PI * M_PI);
    return sigma8 * sigma8 / s2;
}

}  // namespace pmr
