// Internal declarations shared by the host numerics and the CUDA engine.
#pragma once

#include "lexgb.h"

namespace lexgb {

int leja_points(int K, double* xi);
int leja_coeffs(int l, double h, double c, double gamma, const double* xi, int K, double* d);
int leja_coeff_count(double h, double c, double gamma, int K);
// leja_coeffs with caller workspace of 6 * (l + K) doubles (allocates nothing)
int leja_coeffs_ws(int l, double h, double c, double gamma, const double* xi, int K, double* d, double* ws);
// records a message for lx_last_cuda_error() on the calling thread
void set_last_error(const char* msg);

}  // namespace lexgb
