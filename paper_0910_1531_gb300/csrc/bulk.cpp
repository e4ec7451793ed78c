// Bath thermodynamics (App. A): Percus-Yevick hard-sphere chemical potential and
// pressure, and the MSA screening parameter Gamma solved by Newton's method (as App. A
// prescribes), safeguarded by a bracket [0, kappa] on which the equation changes sign.
// The paper's "epsilon" is read as eps0 eps_r throughout, so e^2/(kT eps) = 4 pi lambda_B.
#include "bulk.h"

#include "gb300dft.h"

#include <cmath>

namespace {
constexpr double kE = 1.602176634e-19;       // C
constexpr double kKB = 1.380649e-23;         // J/K
constexpr double kNA = 6.02214076e23;        // 1/mol
constexpr double kEps0 = 8.8541878128e-12;   // F/m
constexpr double kPi = 3.14159265358979323846;

struct Msa {
    int S;
    const double* rho;
    const double* sigma;
    const double* z;
    double delta;   // 1 - xi_3
    double lb;
    // eta(Gamma) and Omega(Gamma) of App. A
    void eta_omega(double g, double* eta, double* omega) const {
        double so = 0.0, se = 0.0;
        for (int j = 0; j < S; ++j) {
            const double d = 1.0 + g * sigma[j];
            so += rho[j] * sigma[j] * sigma[j] * sigma[j] / d;
            se += rho[j] * sigma[j] * z[j] / d;
        }
        *omega = 1.0 + kPi / (2.0 * delta) * so;
        *eta = kPi / (2.0 * delta * (*omega)) * se;
    }
    // F(Gamma) = Gamma^2 - pi lambda_B sum_j rho_j ((z_j - eta sigma_j^2) / (1 + Gamma sigma_j))^2
    double F(double g) const {
        double eta, om;
        eta_omega(g, &eta, &om);
        double s = 0.0;
        for (int j = 0; j < S; ++j) {
            const double t = (z[j] - eta * sigma[j] * sigma[j]) / (1.0 + g * sigma[j]);
            s += rho[j] * t * t;
        }
        return g * g - kPi * lb * s;
    }
};
}  // namespace

// White Bear uniform fluid: Phi = -n0 ln D + n1 n2 / D + n2^3 g(n3) / (36 pi D^2), D = 1 - n3,
// g = (n3 + D^2 ln D) / n3^2 (power series of ln D below n3 = 1/2, where the closed form
// cancels).  beta mu_i = sum_alpha dPhi/dn_alpha w_i^alpha(0) with the fundamental measures
// w_i(0) = (1, R_i, 4 pi R_i^2, 4 pi R_i^3 / 3); beta P = n0 + sum_alpha n_alpha dPhi/dn_alpha - Phi.
static void white_bear_bath(int S, const double* rho, const double* radius, double* mu, double* beta_p) {
    double n[4] = {0, 0, 0, 0};
    for (int j = 0; j < S; ++j) {
        const double R = radius[j];
        n[0] += rho[j];
        n[1] += rho[j] * R;
        n[2] += rho[j] * 4.0 * kPi * R * R;
        n[3] += rho[j] * 4.0 * kPi * R * R * R / 3.0;
    }
    const double D = 1.0 - n[3], lnD = std::log(D);
    double g, dg;
    if (n[3] < 0.5) {
        double sg = 0.0, sd = 0.0;
        for (int k = 60; k >= 3; --k) {
            sg = sg * n[3] + 2.0 / (double(k) * (k - 1) * (k - 2));
            sd = sd * n[3] + 2.0 / (double(k) * (k - 1));
        }
        g = 1.5 - n[3] * sg;
        dg = -sd;
    } else {
        const double num = n[3] + D * D * lnD;
        g = num / (n[3] * n[3]);
        dg = (n[3] - 2.0 * D * lnD) / (n[3] * n[3]) - 2.0 * num / (n[3] * n[3] * n[3]);
    }
    const double f = g / (36.0 * kPi * D * D);
    const double df = (dg * D + 2.0 * g) / (36.0 * kPi * D * D * D);
    const double phi = -n[0] * lnD + n[1] * n[2] / D + n[2] * n[2] * n[2] * f;
    const double d[4] = {-lnD, n[2] / D, n[1] / D + 3.0 * n[2] * n[2] * f,
                         n[0] / D + n[1] * n[2] / (D * D) + n[2] * n[2] * n[2] * df};
    for (int i = 0; i < S; ++i) {
        const double R = radius[i];
        mu[i] = d[0] + d[1] * R + d[2] * 4.0 * kPi * R * R + d[3] * 4.0 * kPi * R * R * R / 3.0;
    }
    *beta_p = n[0] + n[0] * d[0] + n[1] * d[1] + n[2] * d[2] + n[3] * d[3] - phi;
}

bool compute_bath(int S, const double* radius, const double* z, const double* molar, double T, double eps_r,
                  BathState* out, std::string* err, int functional) {
    out->rho.assign(S, 0.0);
    out->mu_hs.assign(S, 0.0);
    out->mu_es.assign(S, 0.0);
    out->lam.assign(S, 0.0);
    out->lb = kE * kE / (4.0 * kPi * kEps0 * eps_r * kKB * T) * 1e9;
    std::vector<double> sigma(S);
    for (int i = 0; i < S; ++i) {
        out->rho[i] = molar[i] * kNA * 1e-24;
        sigma[i] = 2.0 * radius[i];
    }
    // Percus-Yevick / scaled particle (eqs. muHSBath, HSPressure)
    double xi[4] = {0, 0, 0, 0};
    for (int n = 0; n < 4; ++n)
        for (int j = 0; j < S; ++j) xi[n] += kPi / 6.0 * out->rho[j] * std::pow(sigma[j], n);
    const double delta = 1.0 - xi[3];
    out->beta_p = 6.0 / kPi * (xi[0] / delta + 3.0 * xi[1] * xi[2] / (delta * delta)
                               + 3.0 * xi[2] * xi[2] * xi[2] / (delta * delta * delta));
    for (int i = 0; i < S; ++i) {
        const double s = sigma[i];
        out->mu_hs[i] = -std::log(delta) + (3.0 * xi[2] * s + 3.0 * xi[1] * s * s) / delta
                        + 9.0 * xi[2] * xi[2] * s * s / (2.0 * delta * delta) + kPi * out->beta_p * s * s * s / 6.0;
    }
    if (functional == DFT_PHI_WHITE_BEAR) white_bear_bath(S, out->rho.data(), radius, out->mu_hs.data(), &out->beta_p);
    // MSA Gamma (eq. Gamma) by Newton on F with a numerical derivative, kept in [lo, hi]
    double k2 = 0.0;
    for (int j = 0; j < S; ++j) k2 += 4.0 * kPi * out->lb * out->rho[j] * z[j] * z[j];
    const double kappa = std::sqrt(k2);
    Msa m{S, out->rho.data(), sigma.data(), z, delta, out->lb};
    double g = 0.0;
    if (kappa > 0.0) {
        double lo = 0.0, hi = kappa;
        int widen = 0;
        while (m.F(hi) <= 0.0 && widen < 60) { hi *= 2.0; ++widen; }
        if (m.F(hi) <= 0.0) { *err = "MSA Gamma equation has no root"; return false; }
        g = 0.5 * kappa;
        for (int it = 0; it < 200; ++it) {
            const double f = m.F(g);
            if (f < 0.0) lo = g; else hi = g;
            const double h = 1e-7 * (g > 1e-3 ? g : 1e-3);
            const double df = (m.F(g + h) - m.F(g - h)) / (2.0 * h);
            double gn = (df != 0.0) ? g - f / df : 0.5 * (lo + hi);
            if (!(gn > lo && gn < hi)) gn = 0.5 * (lo + hi);
            const double step = std::fabs(gn - g);
            g = gn;
            if (step <= 1e-15 * g || hi - lo <= 1e-15 * hi) break;
        }
    }
    out->gamma = g;
    double eta = 0.0, om = 1.0;
    if (g > 0.0) m.eta_omega(g, &eta, &om);
    for (int i = 0; i < S; ++i) {
        const double s = sigma[i];
        const double d = 1.0 + g * s;
        out->mu_es[i] = -out->lb * (g * z[i] * z[i] / d + eta * s * ((2.0 * z[i] - eta * s * s) / d + eta * s * s / 3.0));
        out->lam[i] = (g > 0.0) ? radius[i] + 0.5 / g : INFINITY;
    }
    return true;
}
