// Host-side FP64 construction of the FMM translation operators (see operators.cpp).
#pragma once
#include <complex>
#include <vector>

namespace fmmcph {

double norm_nm(int n, int m);
void regular_c(const double u[3], int P, std::vector<std::complex<double>>& R);
void irregular_c(const double t[3], int P, std::vector<std::complex<double>>& I);

// Real-form, normalised operators, nc x nc row-major (nc = (P+1)^2).
void op_m2l(int P, const int o[3], double* out);  // source = target + o
void op_m2m(int P, int oct, double* out);         // child octant -> parent
void op_l2l(int P, int oct, double* out);         // parent -> child octant
void op_lattice(int P, double* out);              // periodic far images, root level
void lattice_coefficients(int Q, std::vector<std::complex<double>>& g);
void regular_real_hat(int P, const double u[3], double* out);

}  // namespace fmmcph
