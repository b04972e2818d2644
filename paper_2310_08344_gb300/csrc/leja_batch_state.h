// Per-instance and shared state of the batched Leja loop (leja_batch.cuh,
// and the float-float batch kernel in lexgb_batch_df.cu).
#pragma once

#include <cuda_runtime.h>

namespace lexgb {

struct BatchInst {
  int nx, ny;
  int first_strip, nstrips;
  int kmax;
  int done, status, iters;
  double wxp, wxm, wyp, wym, wc0;
  double rtol, atol;
  const double* w;
  double* y0;
  double* y1;
  double* p;
  const double* d;
  double ynorm, pnorm, err;
  // float-float batches: the basis and the polynomial as float pairs, the
  // hi/lo floats of wxp, wxm, wyp, wym, and the storage scaling of the
  // instance (stored y_m = y_m 2^-sig, p in 2^-kscale units, the next basis
  // vector renormalised by 2^-dlt; wexp: largest biased exponent of |w|)
  float2* yf0;
  float2* yf1;
  float2* pf;
  float wf[8];
  int wexp, kscale, sig, dlt;
  // two iterations per pass: an instance that stopped after the first of
  // them holds p_{m+2}; the output pass subtracts fix_d * (basis fix_buf)
  int fix, fix_buf;
  double fix_d;
};

struct BatchState {
  int m;       // global iteration index
  int active;  // instances not yet done
  int mmax;    // safety cap on m
  int pad;
};

}  // namespace lexgb
