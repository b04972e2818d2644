// Internal declarations shared by the host numerics and the CUDA engine.
#pragma once

#include "lexgb.h"

namespace lexgb {

int leja_points(int K, double* xi);
int leja_coeffs(int l, double h, double c, double gamma, const double* xi, int K, double* d);
int leja_coeff_count(double h, double c, double gamma, int K);

}  // namespace lexgb
