// Host-side helpers of the level setup (implemented in setup_host.cu).
#pragma once
#include <vector>

namespace host {
void gll(int p, std::vector<double>& x, std::vector<double>& w);
std::vector<double> diff_matrix(const std::vector<double>& x);
std::vector<double> interp(const std::vector<double>& x, const std::vector<double>& y);
void trilinear(const double* cr, double x1, double x2, double x3, double X[3], double J[9]);
bool is_box(const double* cr, double h[3]);
double exact_volume(const double* cr);
void surrogate_widths(const double* cr, double dx[3]);
void jacobi_eig(int n, std::vector<double>& A, std::vector<double>& V);
int overlap_layers(int p, double delta);
void fd_variant(int p, int m, double mu_star, double delta, char left, char right,
                std::vector<double>& S, std::vector<double>& lam, std::vector<double>& W);
}  // namespace host
