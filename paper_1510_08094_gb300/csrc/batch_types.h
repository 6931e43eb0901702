// Data of a batched plan shared by the host plan code and the persistent kernel.
#pragma once

#include "fft.cuh"

namespace sp {

struct BatchClass {
  int nt, nl, L, N, K, Kp;
  int rows, cols;                      // transform tiles (rows / columns per pass of the CTA)
  FftDesc row_fft, col_fft;
  const cpx<double>* tw_row;
  const cpx<double>* tw_col;
  const cpx<double>* post_row;
  const cpx<double>* post_col;
  const cpx<double>* post_col_s;       // post_col / (2N), for the forward colatitude transform
  const int* perm_row;
  const int* perm_col;
  const double* row_scale;
  const double* fl;                    // [N][Kp] factorised parity tridiagonals
  const double* fiu;
  const double* fcu;
};

struct BatchProblem {
  int cls;
  int pad;
  long long off;                       // offset of f and u in doubles
};

struct BatchArgs {
  const BatchClass* classes;
  const BatchProblem* problems;
  const int* order;                    // problem indices, largest first
  int count;
  const double* f;
  double* u;
  cpx<double>* scratch;                // gridDim.x slots
  long long slot;                      // complex elements per slot
  int* counter;                        // zeroed before the launch
};

}  // namespace sp
