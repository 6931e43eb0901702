// Data of a batched plan shared by the host plan code and the persistent kernel.
#pragma once

#include "dd.cuh"
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
  const double* fl;                    // [N][Kp] factorised parity tridiagonals (FP64 plans)
  const double* fiu;
  const double* fcu;
  // FP32 + refinement plans: double-float transform tables, FP32 factors of every
  // column, FP64 factors of the k = 0 column ([N][2], column 0 used)
  const cpx<dd>* tw_row_d;
  const cpx<dd>* tw_col_d;
  const cpx<dd>* post_row_d;
  const cpx<dd>* post_col_d;
  const cpx<dd>* post_col_s_d;
  const dd* row_scale_d;
  const float* fl32;                   // [N][Kp]
  const float* fiu32;
  const float* fcu32;
  const double* zl;                    // [N][2]
  const double* ziu;
  const double* zcu;
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
  long long slot;                      // 16-byte units per slot
  int* counter;                        // zeroed before the launch
  int sweeps;                          // refinement sweeps (FP32 + refinement plans)
};

// Pivot record of one step of the structure-preserving GE (written by the
// pivot-search kernels, read by the host).
struct GePivot {
  double best;      // largest sigma_1(M) = max(|a + b|, |a - b|) over the search region
  double a, b;      // the pivot's a = e(lambda* - pi, theta*), b = e(lambda*, theta*)
  double maxabs;    // max |e| over the half grid
  long long index;  // i * (n/2) + (q - n/2) of the pivot (smallest index among ties)
};

// One launch of the tangential coefficient maps: output o receives +-T_c,
// c = comp[o], of the gradient components of one input (c = 0 x, 1 y, 2 z),
// added to its contents when bit o of acc is set.
struct TangentialCombo {
  cpx<double>* G[3];        // outputs (null: unused)
  signed char comp[3];      // component of output o
  unsigned char neg[3];     // output o takes -T_c
  unsigned char acc;        // bit o: output o is added to
  unsigned char need_xy;    // some output uses T0 or T1 (reads Q)
  unsigned char need_z;     // some output uses T2
};

}  // namespace sp
