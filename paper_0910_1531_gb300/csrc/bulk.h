// Bath thermodynamics of App. A on the host, in FP64 (computed once per plan).
#pragma once

#include <string>
#include <vector>

struct BathState {
    std::vector<double> rho;    // nm^-3
    std::vector<double> mu_hs;  // beta mu^{HS,bath}  (eq. muHSBath, or the White Bear uniform limit)
    std::vector<double> mu_es;  // beta mu^{ES,bath}  (MSA, App. A)
    std::vector<double> lam;    // lambda_k = R_k + 1/(2 Gamma)
    double beta_p = 0.0;        // beta P^{HS}_bath (eq. HSPressure), nm^-3
    double gamma = 0.0;         // MSA Gamma (eq. Gamma), nm^-1
    double lb = 0.0;            // Bjerrum length e^2/(4 pi eps0 eps_r kT), nm
};

// Returns false (and a message) if the MSA equation has no root in range.  functional: the
// hard-sphere form (DFT_PHI_*); DFT_PHI_WHITE_BEAR takes mu^HS and P from that form's uniform
// limit instead of App. A's Percus-Yevick expressions.
bool compute_bath(int S, const double* radius, const double* z, const double* molar, double temperature_K,
                  double eps_r, BathState* out, std::string* err, int functional = 0);
