// C ABI of the spherical Poisson solver (declarations and argument rules in
// include/sphere_poisson.h).  Host side: plan construction (FFT radix plans,
// twiddle tables, launch shapes, the factorised per-k tridiagonals) and the
// launch sequences of the solve and of its transpose.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <initializer_list>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "sphere_poisson.h"
#include "launch.h"

using sp::cpx;
using sp::FftDesc;

namespace {

constexpr int kMaxLen = 12288;             // longest transform (n_theta, n_lambda/2)
constexpr size_t kSmemBudget = 200 * 1024;  // shared memory per CTA for a transform tile
constexpr int kBatchThreadsPerCta = 256;     // threads of a persistent batched CTA
constexpr int kHostChunks = 16;              // row chunks of the host-buffer solve's overlapped copies
constexpr double kMeanWarnFactor = 1e3 * 2.220446049250313080847263336181640625e-16;  // 1e3 eps
constexpr uint32_t kMagic = 0x53504f31u;    // "SPO1"
constexpr double kHalfPi = 1.57079632679489661923132169163975144;

thread_local char g_cuda_msg[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_cuda_msg, sizeof g_cuda_msg, "CUDA error in %s: %s", what, cudaGetErrorString(e));
  return SP_ERR_CUDA;
}

#define SP_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Radix plan of a transform length: 8s, then 4 or 2 for the leftover power of
// two, then 5, 3 and the odd primes up to 31.  Returns false if L has a prime
// factor above 31 or needs too many passes.
bool make_fft_desc(int L, FftDesc* d) {
  std::memset(d, 0, sizeof *d);
  d->L = L;
  int rest = L, s = 0;
  auto push = [&](int r) {
    if (s >= sp::kMaxStages) return false;
    d->radix[s++] = r;
    rest /= r;
    return true;
  };
  // odd radices first: the first pass (sub-DFT length 1) reads each
  // butterfly's R inputs R elements apart, which for R = 8 puts a warp's
  // accesses on a few shared-memory banks; odd strides spread them (and the
  // digit-reversed load scatter then steps by L/8 elements, also spread)
  const int primes[] = {5, 3, 7, 11, 13, 17, 19, 23, 29, 31};
  for (int p : primes)
    while (rest % p == 0) if (!push(p)) return false;
  while (rest % 8 == 0) if (!push(8)) return false;
  if (rest % 4 == 0 && !push(4)) return false;
  if (rest % 2 == 0 && !push(2)) return false;
  d->nstages = s;
  d->div_L = sp::make_fastdiv((unsigned)L);
  int ns = 1, off = 0;
  for (int t = 0; t < s; ++t) {
    d->div_nb[t] = sp::make_fastdiv((unsigned)(L / d->radix[t]));
    d->div_ns[t] = sp::make_fastdiv((unsigned)ns);
    d->tw_off[t] = off;
    off += ns * ((d->radix[t] + 1) & ~1);
    ns *= d->radix[t];
  }
  for (int t = 0; t < s; ++t) {
    const int R = d->radix[t];
    if (R >= 7 && (R & 1)) {
      d->dft_off[t] = off;
      off += (R + 1) & ~1;
    }
  }
  ns = 1;
  for (int t = 0; t < s; ++t) {
    d->g_off[t] = -1;
    const int rt = d->radix[t];
    if ((rt == 2 || rt == 3 || rt == 4 || rt == 5 || rt == 8) && ns > 1) {
      static_assert(sizeof(sp::Radix5Record) == sizeof(sp::Radix8Record) &&
                    sizeof(sp::Radix5Record) == sizeof(sp::Radix4Record) &&
                    sizeof(sp::Radix5Record) == sizeof(sp::Radix3Record) &&
                    sizeof(sp::Radix5Record) == sizeof(sp::Radix2Record), "one record size");
      d->g_off[t] = off;
      off += ns * (int)(sizeof(sp::Radix5Record) / sizeof(cpx<double>));
    }
    ns *= d->radix[t];
  }
  d->tw_len = off;
  return rest == 1;
}

// threads for a CTA that transforms nbatch sequences of the plan's length:
// about one butterfly of the smallest radix per thread, 64 .. 512 (64 .. 256
// for the large-prime kernels, whose launch bound is 256 threads)
int fft_threads(const FftDesc& d, int nbatch) {
  int rmin = 32;
  bool big = false;
  for (int s = 0; s < d.nstages; ++s) {
    rmin = d.radix[s] < rmin ? d.radix[s] : rmin;
    big = big || d.radix[s] > 8;
  }
  const long cap = big ? 256 : 512;
  long want = (long)nbatch * d.L / rmin;
  int t = (int)(want < 64 ? 64 : (want > cap ? cap : want));
  return (t + 31) / 32 * 32;
}

// mixed-radix digit reversal for the in-place decimation-in-time passes:
// q = r_1 + R_s (r_2 + R_{s-1} (r_3 + ...)) goes to p = r_1 L/R_s + r_2 L/(R_s R_{s-1}) + ...
void digit_reversal(const FftDesc& d, std::vector<int>& perm) {
  perm.resize(d.L);
  for (int q0 = 0; q0 < d.L; ++q0) {
    int q = q0, p = 0, w = d.L;
    for (int s = d.nstages - 1; s >= 0; --s) {
      int R = d.radix[s];
      w /= R;
      p += (q % R) * w;
      q /= R;
    }
    perm[q0] = p;
  }
}

// exp(-2 pi i t / M), with the angle reduced exactly: 4t = q M + r, |r| <= M/2,
// so 2 pi t/M = q pi/2 + (pi/2) r/M and the residual angle is within +-pi/4.
void unit_root(long t, long M, double* re, double* im) {
  t %= M;
  if (t < 0) t += M;
  long q = (4 * t + M / 2) / M;  // nearest quarter turn
  long r = 4 * t - q * M;
  double phi = kHalfPi * (double)r / (double)M;
  double c = std::cos(phi), s = std::sin(phi);
  // angle = q pi/2 + phi; value exp(-i angle)
  double cr, sr;
  switch (q & 3) {
    case 0: cr = c; sr = s; break;
    case 1: cr = -s; sr = c; break;
    case 2: cr = -c; sr = -s; break;
    default: cr = s; sr = -c; break;
  }
  *re = cr;
  *im = -sr;
}

// the twiddle table of an FFT descriptor (layout in FftDesc)
std::vector<cpx<double>> stage_twiddles(const FftDesc& d) {
  std::vector<cpx<double>> tab(d.tw_len, cpx<double>{1.0, 0.0});
  int ns = 1;
  for (int s = 0; s < d.nstages; ++s) {
    const int R = d.radix[s], RP = (R + 1) & ~1;
    for (int k = 0; k < ns; ++k)
      for (int r = 0; r < R; ++r) {
        cpx<double>& w = tab[d.tw_off[s] + k * RP + r];
        unit_root((long)r * k, (long)ns * R, &w.re, &w.im);
      }
    if (R >= 7 && (R & 1))
      for (int a = 0; a < R; ++a) unit_root(a, R, &tab[d.dft_off[s] + a].re, &tab[d.dft_off[s] + a].im);
    // w_r = sigma_r (1 + i tau_r), or i sigma_r (1 + i tau_r) where |Im w_r| > |Re w_r|
    auto scaled_root = [&](int r, int k, double* sigma, double* tau, long long* rot) {
      double re, im;
      unit_root((long)r * k, (long)ns * R, &re, &im);
      if (std::fabs(re) >= std::fabs(im)) {
        *sigma = re;
        *tau = im / re;
      } else {
        *sigma = im;
        *tau = -re / im;
        *rot |= 1LL << (r - 1);
      }
    };
    if (d.g_off[s] >= 0 && R == 8) {
      const size_t per = sizeof(sp::Radix8Record) / sizeof(cpx<double>);
      for (int k = 0; k < ns; ++k) {
        sp::Radix8Record rec = {};
        double sg[8] = {1.0};
        for (int r = 1; r < 8; ++r) scaled_root(r, k, &sg[r], &rec.tau[r - 1], &rec.rot);
        rec.s4 = sg[4];
        rec.q62 = sg[6] / sg[2];
        rec.s2 = sg[2];
        rec.q51 = sg[5] / sg[1];
        rec.q73 = sg[7] / sg[3];
        rec.q31 = sg[3] / sg[1];
        rec.s1 = sg[1];
        rec.s1h = 0.70710678118654752440084436210484903928 * sg[1];
        std::memcpy(&tab[d.g_off[s] + k * per], &rec, sizeof rec);
      }
    }
    if (d.g_off[s] >= 0 && R == 4) {
      for (int k = 0; k < ns; ++k) {
        sp::Radix4Record rec = {};
        double sg[4] = {1.0};
        for (int r = 1; r < 4; ++r) scaled_root(r, k, &sg[r], &rec.tau[r - 1], &rec.rot);
        rec.s2 = sg[2];
        rec.q31 = sg[3] / sg[1];
        rec.s1 = sg[1];
        std::memcpy(&tab[d.g_off[s] + k * (sizeof(rec) / sizeof(cpx<double>))], &rec, sizeof rec);
      }
    }
    if (d.g_off[s] >= 0 && R == 3) {
      for (int k = 0; k < ns; ++k) {
        sp::Radix3Record rec = {};
        double sg[3] = {1.0};
        for (int r = 1; r < 3; ++r) scaled_root(r, k, &sg[r], &rec.tau[r - 1], &rec.rot);
        rec.q21 = sg[2] / sg[1];
        rec.s1 = sg[1];
        rec.s1half = 0.5 * sg[1];
        rec.ss1 = 0.86602540378443864676372317075293618347 * sg[1];   // sin(2 pi/3)
        std::memcpy(&tab[d.g_off[s] + k * (sizeof(rec) / sizeof(cpx<double>))], &rec, sizeof rec);
      }
    }
    if (d.g_off[s] >= 0 && R == 2) {
      for (int k = 0; k < ns; ++k) {
        sp::Radix2Record rec = {};
        double sg1 = 1.0;
        scaled_root(1, k, &sg1, &rec.tau, &rec.rot);
        rec.s1 = sg1;
        std::memcpy(&tab[d.g_off[s] + k * (sizeof(rec) / sizeof(cpx<double>))], &rec, sizeof rec);
      }
    }
    if (d.g_off[s] >= 0 && R == 5) {
      // the FP64 radix-5 records
      const double q5 = 0.55901699437494742410229341718281905886;   // sqrt5 / 4
      const double sn1 = 0.95105651629515357211643933337938214340;  // sin(2 pi/5)
      const double sn2 = 0.58778525229247312916870595463907276860;  // sin(4 pi/5)
      const double r5 = 0.61803398874989484820458683436563811772;   // sn2 / sn1
      const double ri5 = 1.61803398874989484820458683436563811772;  // sn1 / sn2
      for (int k = 0; k < ns; ++k) {
        sp::Radix5Record rec = {};
        double sg[4];
        for (int r = 1; r <= 4; ++r) scaled_root(r, k, &sg[r - 1], &rec.tau[r - 1], &rec.rot);
        rec.q4 = sg[3] / sg[0];
        rec.q3 = sg[2] / sg[1];
        rec.rho = sg[1] / sg[0];
        rec.s1 = sg[0];
        rec.s1q = 0.25 * sg[0];
        rec.q5s1 = q5 * sg[0];
        rec.rrho = r5 * rec.rho;
        rec.rirho = ri5 * rec.rho;
        rec.ss1 = sn1 * sg[0];
        rec.ss2 = sn2 * sg[0];
        std::memcpy(&tab[d.g_off[s] + k * (sizeof(rec) / sizeof(cpx<double>))], &rec, sizeof rec);
      }
    }
    ns *= R;
  }
  return tab;
}

}  // namespace

struct sp_plan_s {
  uint32_t magic;
  int nt, nl, L, N, K, Kp;
  int precision, sweeps;
  int device;
  FftDesc row_fft, col_fft;
  bool big_row, big_col;
  // the grid with both poles (SP_FLAG_POLES): nt = N + 1 sample rows, the
  // colatitude transforms of length 2N (poles.cuh)
  bool poles;
  FftDesc pole_fft;
  bool big_pole;
  int pole_threads;
  size_t pole_smem;
  cpx<double>* tw_pole;  // twiddles of the length-2N passes
  int* perm_pole;        // their digit reversal
  int rows_per_cta, cols_per_cta;  // transform tiles in the plan's arithmetic
  bool pipe_rows, pipe_cols;       // pipelined kernels wanted for the row / column stages
  bool pipe[4];                    // pipelined kernel per stage (rows fwd, theta fwd, theta inv, rows inv)
  int pgrid[4];                    // its persistent grid
  size_t psmem[4];                 // its dynamic shared memory
  int row_threads, col_threads;
  size_t row_smem, col_smem;
  int zcol_threads;                // FP64 zonal side path: one column per CTA
  size_t zcol_smem;
  size_t ws_bytes;
  size_t off_x, off_y, off_z;      // workspace layout (bytes): main array at 0
  void* dev;                       // one allocation holding every table
  // double tables (FP64 path and the FP64 zonal side path)
  cpx<double>* tw_row;   // FFT twiddles of the rows (length L, layout in FftDesc)
  cpx<double>* tw_col;   // FFT twiddles of the columns (length N)
  cpx<double>* post_row; // exp(-2 pi i k/n), k <= L
  cpx<double>* post_col; // exp(-i pi j/(2N)), j <= N
  cpx<double>* post_col_s; // the same times 1/(2N) (forward colatitude transform)
  int* perm_row;         // digit reversal of the length-L passes
  int* perm_col;         // digit reversal of the length-N passes
  double* row_scale;     // sin^2(theta_i)/n
  double* row_plain;     // 1/n (transforms without the sin^2 weight)
  double* sin2;          // sin^2(theta_i) (the low-rank right-hand side)
  double* geo;           // sin, cos theta_i; cos, sin lambda_q (the unit normal on the grid)
  double* mean_w;        // w_i / n: the quadrature weight of row i in the mean of f (single plans)
  int sms;               // multiprocessors of the plan's device
  int* dev_status;       // device status word: nonzero when a kernel's bounded wait gave up (read by the host)
  double chop;           // relative coefficient threshold of the derivative operators (0: off)
  void* row_scale_t;     // the same in float (SP_FP32) or double-float (SP_FP32_REFINE)
  // the same tables in float (SP_FP32) or double-float (SP_FP32_REFINE)
  void* tw_row_t;
  void* tw_col_t;
  void* post_row_t;
  void* post_col_t;
  void* post_col_s_t;    // post_col_s in the plan's arithmetic
  // factorised parity tridiagonals l, 1/u, c/u: FP64 [N][Kp] (SP_FP64),
  // float [N][Kp] (FP32 forms) and FP64 [N][2] for the zonal column (FP32 forms)
  double* fac_l;
  double* fac_iu;
  double* fac_cu;
  float* f32_l;
  float* f32_iu;
  float* f32_cu;
  double* z_l;
  double* z_iu;
  double* z_cu;
  // SP_FP32 forward solve and SP_FP32_REFINE solve: the fused colatitude
  // stage (fused.cuh, fused_refine.cuh) and the pivots 1/u of its top-down
  // factorisation, per column [k][j]
  bool fused;
  int fuse_cols, fuse_threads;
  size_t fuse_smem;
  float* fc_iu;
  // the FP32 forms run the zonal column on a second stream
  cudaStream_t side;
  cudaEvent_t ev_fork, ev_join;
  // host-buffer solve: copy stream, a second compute stream for alternate row
  // chunks, and per-chunk events (created on first use)
  cudaStream_t copy, alt;
  std::vector<cudaEvent_t> ov_events;
  // stage timing (profile_begin / profile_end)
  std::vector<cudaEvent_t> prof_events;
  int prof_max, prof_count;
  // batched plans
  int batched;
  int count;
  size_t total;                      // doubles in the packed f / u arrays
  std::vector<size_t> offsets;       // count + 1
  sp::BatchArgs bargs;               // device pointers (f, u, scratch, counter filled per call)
  bool bbig;                         // some class needs the large-prime passes
  // The problems are launched in two groups, each a persistent kernel with its
  // own work counter: the classes whose transforms use radices <= 8 only
  // (order[0 .. bsplit), a kernel fitting two CTAs per SM) and those that need
  // the large-prime passes (order[bsplit .. count), one CTA per SM).
  int bsplit;
  int bgrid_g[2];
  size_t bsmem_g[2];
  int bgrid, bthreads;               // bgrid: the larger group grid (scratch slots)
  size_t bsmem;
  size_t off_counter;                // two counters in the workspace
};

namespace {

bool plan_ok(sp_plan_t p) { return p != nullptr && p->magic == kMagic; }

// SP_OK if the current device is the plan's (its tables live there), else SP_ERR_BAD_ARG
int on_plan_device(sp_plan_t p) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  return dev == p->device ? SP_OK : SP_ERR_BAD_ARG;
}

// Reads and clears the plan's device status word after `st` has been
// synchronised by the caller: SP_ERR_TIMEOUT if a kernel's bounded wait gave up.
int take_device_status(sp_plan_t p, cudaStream_t st) {
  if (!p->dev_status) return SP_OK;
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, p->dev_status, sizeof v, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "device status read");
  if (v == 0) return SP_OK;
  e = cudaMemsetAsync(p->dev_status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "device status clear");
  return SP_ERR_TIMEOUT;
}

int check_arrays(sp_plan_t p, const void* a, const void* b, const void* ws, size_t ws_bytes) {
  if (!plan_ok(p)) return SP_ERR_BAD_PLAN;
  if (!a || !b || !ws) return SP_ERR_NULL;
  if (((uintptr_t)a | (uintptr_t)b | (uintptr_t)ws) & 15) return SP_ERR_MISALIGNED;
  if (ws_bytes < p->ws_bytes) return SP_ERR_WORKSPACE;
  return on_plan_device(p);
}

// the mean of f and max |f| by the row-weight quadrature: partial sums in the
// first nparts 16-byte slots of the workspace (nparts + 1 slots fit in any
// plan's workspace), the result to `mean` / `absmax` (device; either may be NULL)
int mean_parts(sp_plan_t p) {
  size_t slots = p->ws_bytes / sizeof(double2);
  int n = std::min(p->nt, 2 * std::max(p->sms, 1));
  if (slots < 2) return 0;
  if ((size_t)n > slots - 1) n = (int)(slots - 1);
  return n;
}
int enqueue_mean(sp_plan_t p, const double* f, void* ws, double* mean, double* absmax, cudaStream_t st) {
  const int nparts = mean_parts(p);
  if (nparts < 1) return SP_ERR_WORKSPACE;
  sp::launch_mean(st, f, p->nt, p->nl, p->mean_w, static_cast<double2*>(ws), nparts, mean, absmax);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SP_OK : cuda_fail(e, "mean launch");
}

// true if the radix plan needs the general (large odd prime) pass set
bool needs_big(const FftDesc& d) {
  for (int s = 0; s < d.nstages; ++s)
    if (d.radix[s] > 8) return true;
  return false;
}

constexpr int kStages = 5;
const char* const kStageNames[kStages] = {"rows_forward", "theta_forward", "solve", "theta_inverse",
                                          "rows_inverse"};
// plans whose forward solve runs the fused colatitude stage: stage 1 times the
// fused kernel, stages 2 and 3 are empty
const char* const kFusedStageNames[kStages] = {"rows_forward", "theta_fused", "solve (in theta_fused)",
                                               "theta_inverse (in theta_fused)", "rows_inverse"};

// the fused stage's tile: `cols` columns per CTA and `threads` threads (false
// if its shared memory does not fit)
bool set_fused_tile(sp_plan_t p, int cols, int threads);

// records the boundary event s of the current profiled call, if any
struct StageMarks {
  sp_plan_t p;
  cudaStream_t st;
  bool on;
  void mark(int s) {
    if (on) cudaEventRecord(p->prof_events[(size_t)p->prof_count * (kStages + 1) + s], st);
  }
  void done() {
    if (on) p->prof_count++;
  }
};

size_t esize(int precision) {
  return precision == SP_FP32 ? sizeof(cpx<float>) : sizeof(cpx<double>);
}

template <typename T>
cudaError_t pipe_occupancy_of(int stage, int threads, size_t smem, int* bps) {
  return sp::pipe_occupancy<T>(stage, false, threads, smem, bps);
}

// Decide per stage whether the pipelined kernel runs (wanted, no large-prime
// radix, FFT buffer + staged input within shared memory, at least one CTA per
// SM fits) and size its persistent grid: resident CTAs, at most one per tile.
cudaError_t configure_pipes(sp_plan_t p) {
  const size_t csz = esize(p->precision);
  auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const size_t rbuf = al((size_t)p->rows_per_cta * p->L * csz), cbuf = al((size_t)p->cols_per_cta * p->N * csz);
  const size_t need[4] = {rbuf + (size_t)p->rows_per_cta * p->nl * sizeof(double),
                          cbuf + (size_t)p->N * p->cols_per_cta * csz, cbuf + (size_t)p->N * p->cols_per_cta * csz,
                          rbuf + (size_t)p->rows_per_cta * p->Kp * csz};
  const bool want[4] = {p->pipe_rows && !p->big_row, p->pipe_cols && !p->big_col, p->pipe_cols && !p->big_col,
                        p->pipe_rows && !p->big_row};
  const int threads[4] = {p->row_threads, p->col_threads, p->col_threads, p->row_threads};
  const int rt = (p->nt + p->rows_per_cta - 1) / p->rows_per_cta, ct = (p->K + p->cols_per_cta - 1) / p->cols_per_cta;
  const int ntiles[4] = {rt, ct, ct, rt};
  int sms = 1;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) return e;
  for (int s = 0; s < 4; ++s) {
    p->pipe[s] = false;
    if (!want[s] || need[s] > 220 * 1024) continue;
    int bps = 0;
    if (p->precision == SP_FP64) e = pipe_occupancy_of<double>(s, threads[s], need[s], &bps);
    else if (p->precision == SP_FP32) e = pipe_occupancy_of<float>(s, threads[s], need[s], &bps);
    else e = pipe_occupancy_of<sp::dd>(s, threads[s], need[s], &bps);
    if (e != cudaSuccess) return e;
    if (bps < 1) continue;
    p->pipe[s] = true;
    p->pgrid[s] = std::max(1, std::min(ntiles[s], sms * bps));
    p->psmem[s] = need[s];
  }
  return cudaSuccess;
}

// The transform launches of a plan: the pipelined persistent kernel where the
// plan chose it for that stage (pipe[s], grid pgrid[s], shared memory psmem[s]),
// else one CTA per tile.
template <typename T>
void launch_rows_forward_x(sp_plan_t p, bool adj, cudaStream_t st, const double* f, cpx<T>* W, int nt, int n,
                           int Kp, int rows, const FftDesc& d, const cpx<T>* tw, const int* perm,
                           const cpx<T>* post, const double* rs, const T* rst, cpx<double>* zonal) {
  if (p->pipe[0])
    sp::launch_rows_forward_pipe<T>(adj, sp::Launch{dim3(p->pgrid[0]), p->row_threads, p->psmem[0], st}, f, W, nt,
                                    n, Kp, rows, d, tw, perm, post, rs, rst, zonal);
  else
    sp::launch_rows_forward<T>(adj, p->big_row,
                               sp::Launch{dim3((nt + rows - 1) / rows), p->row_threads, p->row_smem, st}, f, W, nt,
                               n, Kp, rows, d, tw, perm, post, rs, rst, zonal);
}
template <typename T>
void launch_theta_forward_x(sp_plan_t p, bool adj, cudaStream_t st, cpx<T>* W, int N, int K, int Kp, int cols,
                            const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post, T inv_n,
                            int zonal) {
  if (p->pipe[1])
    sp::launch_theta_forward_pipe<T>(adj, sp::Launch{dim3(p->pgrid[1]), p->col_threads, p->psmem[1], st}, W, N, K,
                                     Kp, cols, d, tw, perm, post, inv_n, zonal);
  else
    sp::launch_theta_forward<T>(adj, p->big_col,
                                sp::Launch{dim3((K + cols - 1) / cols), p->col_threads, p->col_smem, st}, W, N, K,
                                Kp, cols, d, tw, perm, post, inv_n, zonal);
}
template <typename T>
void launch_theta_inverse_x(sp_plan_t p, bool adj, cudaStream_t st, cpx<T>* W, int N, int K, int Kp, int cols,
                            const FftDesc& d, const cpx<T>* tw, const int* perm, const cpx<T>* post, T inv_n,
                            int zonal) {
  if (p->pipe[2])
    sp::launch_theta_inverse_pipe<T>(adj, sp::Launch{dim3(p->pgrid[2]), p->col_threads, p->psmem[2], st}, W, N, K,
                                     Kp, cols, d, tw, perm, post, inv_n, zonal);
  else
    sp::launch_theta_inverse<T>(adj, p->big_col,
                                sp::Launch{dim3((K + cols - 1) / cols), p->col_threads, p->col_smem, st}, W, N, K,
                                Kp, cols, d, tw, perm, post, inv_n, zonal);
}
template <typename T>
void launch_rows_inverse_x(sp_plan_t p, bool adj, cudaStream_t st, const cpx<T>* W, double* u, int nt, int n,
                           int Kp, int rows, const FftDesc& d, const cpx<T>* tw, const int* perm,
                           const cpx<T>* post, const double* rs, const T* rst, const cpx<double>* zonal) {
  if (p->pipe[3])
    sp::launch_rows_inverse_pipe<T>(adj, sp::Launch{dim3(p->pgrid[3]), p->row_threads, p->psmem[3], st}, W, u, nt,
                                    n, Kp, rows, d, tw, perm, post, rs, rst, zonal);
  else
    sp::launch_rows_inverse<T>(adj, p->big_row,
                               sp::Launch{dim3((nt + rows - 1) / rows), p->row_threads, p->row_smem, st}, W, u, nt,
                               n, Kp, rows, d, tw, perm, post, rs, rst, zonal);
}

// Host-buffer solve with the copies overlapped: the grid moves in row chunks on
// the plan's copy stream; the longitude forward transform of chunk c starts as
// soon as its rows have arrived, and the rows of u go back chunk by chunk as
// the longitude inverse transform finishes them.  Consecutive chunks' transforms
// alternate between the solve's stream and a second one, so that one chunk's
// last CTAs run beside the next chunk's first ones instead of leaving the SMs
// idle at every chunk boundary.
struct HostOverlap {
  const double* f_host;
  double* u_host;
  double* d_f;
  double* d_u;
  cudaStream_t copy;
  cudaStream_t alt;
  const cudaEvent_t* ev_in;   // one per chunk
  const cudaEvent_t* ev_out;  // one per chunk
  const cudaEvent_t* ev_sync; // fork / join of alt for the two stages (4)
  int chunks;
};

int overlap_chunk_rows(sp_plan_t p, const HostOverlap* ov) { return (p->nt + ov->chunks - 1) / ov->chunks; }

template <typename T>
void rows_forward_stage(sp_plan_t p, bool adj, cudaStream_t st, const double* in, cpx<T>* W, const cpx<T>* tw,
                        const cpx<T>* post, const double* rs, const T* rst, cpx<double>* zonal,
                        const HostOverlap* ov) {
  if (!ov) {
    launch_rows_forward_x<T>(p, adj, st, in, W, p->nt, p->nl, p->Kp, p->rows_per_cta, p->row_fft, tw,
                             p->perm_row, post, rs, rst, zonal);
    return;
  }
  const int chunk = overlap_chunk_rows(p, ov);
  cudaEventRecord(ov->ev_sync[0], st);
  cudaStreamWaitEvent(ov->alt, ov->ev_sync[0], 0);
  for (int c = 0, r0 = 0; r0 < p->nt; ++c, r0 += chunk) {
    const int nr = std::min(chunk, p->nt - r0);
    const size_t off = (size_t)r0 * p->nl;
    cudaStream_t sc = (c & 1) ? ov->alt : st;
    cudaMemcpyAsync(ov->d_f + off, ov->f_host + off, (size_t)nr * p->nl * sizeof(double), cudaMemcpyHostToDevice,
                    ov->copy);
    cudaEventRecord(ov->ev_in[c], ov->copy);
    cudaStreamWaitEvent(sc, ov->ev_in[c], 0);
    launch_rows_forward_x<T>(p, adj, sc, ov->d_f + off, W + (size_t)r0 * p->Kp, nr, p->nl, p->Kp,
                             p->rows_per_cta, p->row_fft, tw, p->perm_row, post, rs + r0, rst + r0,
                             zonal ? zonal + 2 * (size_t)r0 : nullptr);
  }
  cudaEventRecord(ov->ev_sync[1], ov->alt);
  cudaStreamWaitEvent(st, ov->ev_sync[1], 0);
}

template <typename T>
void rows_inverse_stage(sp_plan_t p, bool adj, cudaStream_t st, const cpx<T>* W, double* out, const cpx<T>* tw,
                        const cpx<T>* post, const double* rs, const T* rst, const cpx<double>* zonal,
                        const HostOverlap* ov) {
  if (!ov) {
    launch_rows_inverse_x<T>(p, adj, st, W, out, p->nt, p->nl, p->Kp, p->rows_per_cta, p->row_fft, tw,
                             p->perm_row, post, rs, rst, zonal);
    return;
  }
  const int chunk = overlap_chunk_rows(p, ov);
  cudaEventRecord(ov->ev_sync[2], st);
  cudaStreamWaitEvent(ov->alt, ov->ev_sync[2], 0);
  for (int c = 0, r0 = 0; r0 < p->nt; ++c, r0 += chunk) {
    const int nr = std::min(chunk, p->nt - r0);
    const size_t off = (size_t)r0 * p->nl;
    cudaStream_t sc = (c & 1) ? ov->alt : st;
    launch_rows_inverse_x<T>(p, adj, sc, W + (size_t)r0 * p->Kp, ov->d_u + off, nr, p->nl, p->Kp,
                             p->rows_per_cta, p->row_fft, tw, p->perm_row, post, rs + r0, rst + r0,
                             zonal ? zonal + 2 * (size_t)r0 : nullptr);
    cudaEventRecord(ov->ev_out[c], sc);
    cudaStreamWaitEvent(ov->copy, ov->ev_out[c], 0);
    cudaMemcpyAsync(ov->u_host + off, ov->d_u + off, (size_t)nr * p->nl * sizeof(double), cudaMemcpyDeviceToHost,
                    ov->copy);
  }
  cudaEventRecord(ov->ev_sync[3], ov->alt);
  cudaStreamWaitEvent(st, ov->ev_sync[3], 0);
}

void enqueue_fp64(sp_plan_t p, bool adj, const double* in, double* out, void* ws, cudaStream_t st,
                  const HostOverlap* ov = nullptr) {
  using sp::Launch;
  cpx<double>* W = static_cast<cpx<double>*>(ws);
  StageMarks m{p, st, !p->prof_events.empty() && p->prof_count < p->prof_max};
  const Launch solve{dim3((p->K + 31) / 32, 2), 32, 0, st};
  const double inv_n = 1.0 / (double)p->N;
  m.mark(0);
  rows_forward_stage<double>(p, adj, st, in, W, p->tw_row, p->post_row, p->row_scale, p->row_scale, nullptr, ov);
  m.mark(1);
  const Launch pole{dim3(p->K), p->pole_threads, p->pole_smem, st};
  if (p->poles && adj)
    sp::launch_theta_poles_adj(false, p->big_pole, pole, W, p->N, p->K, p->Kp, p->pole_fft, p->tw_pole,
                               p->perm_pole);
  else if (p->poles)
    sp::launch_theta_poles(false, p->big_pole, pole, W, p->N, p->K, p->Kp, p->pole_fft, p->tw_pole, p->perm_pole);
  else
    launch_theta_forward_x<double>(p, adj, st, W, p->N, p->K, p->Kp, p->cols_per_cta, p->col_fft,
                                     p->tw_col, p->perm_col, adj ? p->post_col : p->post_col_s, inv_n, 1);
  m.mark(2);
  sp::launch_solve<double>(adj, solve, W, p->fac_l, p->fac_iu, p->fac_cu, p->N, p->K, p->Kp);
  m.mark(3);
  if (p->poles && adj)
    sp::launch_theta_poles_adj(true, p->big_pole, pole, W, p->N, p->K, p->Kp, p->pole_fft, p->tw_pole,
                               p->perm_pole);
  else if (p->poles)
    sp::launch_theta_poles(true, p->big_pole, pole, W, p->N, p->K, p->Kp, p->pole_fft, p->tw_pole, p->perm_pole);
  else
    launch_theta_inverse_x<double>(p, adj, st, W, p->N, p->K, p->Kp, p->cols_per_cta, p->col_fft,
                                     p->tw_col, p->perm_col, p->post_col, inv_n, 1);
  m.mark(4);
  rows_inverse_stage<double>(p, adj, st, W, out, p->tw_row, p->post_row, p->row_scale, p->row_scale, nullptr, ov);
  m.mark(5);
  m.done();
}

// FP64 transforms and eliminations of the zonal column Z [N][2] (one column)
void enqueue_zonal_fp64(sp_plan_t p, bool adj, cpx<double>* Z, cudaStream_t st) {
  const double inv_n = 1.0 / (double)p->N;
  const sp::Launch one{dim3(1), p->zcol_threads, p->zcol_smem, st};
  sp::launch_theta_forward<double>(adj, p->big_col, one, Z, p->N, 1, 2, 1, p->col_fft, p->tw_col, p->perm_col,
                                   adj ? p->post_col : p->post_col_s, inv_n, 1);
  sp::launch_zonal_scan(adj, st, Z, p->z_l, p->z_iu, p->z_cu, p->N);
  sp::launch_theta_inverse<double>(adj, p->big_col, one, Z, p->N, 1, 2, 1, p->col_fft, p->tw_col, p->perm_col,
                                   p->post_col, inv_n, 1);
}

void enqueue_fp32(sp_plan_t p, bool adj, const double* in, double* out, void* ws, cudaStream_t st,
                  const HostOverlap* ov = nullptr) {
  using sp::Launch;
  cpx<float>* W = static_cast<cpx<float>*>(ws);
  cpx<double>* Z = reinterpret_cast<cpx<double>*>(static_cast<char*>(ws) + p->off_z);
  StageMarks m{p, st, !p->prof_events.empty() && p->prof_count < p->prof_max};
  const Launch solve{dim3((p->K + 31) / 32, 2), 32, 0, st};
  const float inv_n = 1.0f / (float)p->N;
  const cpx<float>* twr = static_cast<const cpx<float>*>(p->tw_row_t);
  const cpx<float>* twc = static_cast<const cpx<float>*>(p->tw_col_t);
  const cpx<float>* por = static_cast<const cpx<float>*>(p->post_row_t);
  const cpx<float>* poc = static_cast<const cpx<float>*>(p->post_col_t);
  m.mark(0);
  rows_forward_stage<float>(p, adj, st, in, W, twr, por, p->row_scale, static_cast<const float*>(p->row_scale_t),
                            Z, ov);
  cudaEventRecord(p->ev_fork, st);
  cudaStreamWaitEvent(p->side, p->ev_fork, 0);
  enqueue_zonal_fp64(p, adj, Z, p->side);
  cudaEventRecord(p->ev_join, p->side);
  m.mark(1);
  if (!adj && p->fused) {
    sp::launch_theta_fused(p->big_col,
                           Launch{dim3((p->K + std::max(p->fuse_cols, 1) - 1) / std::max(p->fuse_cols, 1)),
                                  p->fuse_threads, p->fuse_smem, st},  // grid recomputed for cols <= 0
                           W, p->N, p->K, p->Kp, p->fuse_cols, p->col_fft, twc, p->perm_col,
                           static_cast<const cpx<float>*>(p->post_col_s_t), poc, p->fc_iu, inv_n, p->dev_status);
    m.mark(2);
    m.mark(3);
  } else if (adj && p->fused && p->fuse_cols < 0) {
    // the adjoint's colatitude stage in one launch, on the forward's single-buffer tile
    sp::launch_theta_fused_adj(p->big_col, Launch{dim3(1), p->fuse_threads, p->fuse_smem, st}, W, p->N, p->K,
                               p->Kp, p->fuse_cols, p->col_fft, twc, p->perm_col, poc, p->fc_iu, inv_n,
                               p->dev_status);
    m.mark(2);
    m.mark(3);
  } else {
    launch_theta_forward_x<float>(p, adj, st, W, p->N, p->K, p->Kp, p->cols_per_cta, p->col_fft,
                                    twc, p->perm_col, adj ? poc : static_cast<const cpx<float>*>(p->post_col_s_t),
                                    inv_n, 0);
    m.mark(2);
    sp::launch_solve<float>(adj, solve, W, p->f32_l, p->f32_iu, p->f32_cu, p->N, p->K, p->Kp);
    m.mark(3);
    launch_theta_inverse_x<float>(p, adj, st, W, p->N, p->K, p->Kp, p->cols_per_cta, p->col_fft,
                                    twc, p->perm_col, poc, inv_n, 0);
  }
  cudaStreamWaitEvent(st, p->ev_join, 0);
  m.mark(4);
  rows_inverse_stage<float>(p, adj, st, W, out, twr, por, p->row_scale, static_cast<const float*>(p->row_scale_t),
                            Z, ov);
  m.mark(5);
  m.done();
}

void enqueue_refine(sp_plan_t p, const double* in, double* out, void* ws, cudaStream_t st,
                    const HostOverlap* ov = nullptr) {
  using sp::Launch;
  using sp::dd;
  char* base = static_cast<char*>(ws);
  cpx<dd>* Fd = reinterpret_cast<cpx<dd>*>(base);
  cpx<dd>* Xd = reinterpret_cast<cpx<dd>*>(base + p->off_x);
  cpx<float>* Y = reinterpret_cast<cpx<float>*>(base + p->off_y);
  cpx<double>* Z = reinterpret_cast<cpx<double>*>(base + p->off_z);
  StageMarks m{p, st, !p->prof_events.empty() && p->prof_count < p->prof_max};
  const Launch solve{dim3((p->K + 31) / 32, 2), 32, 0, st};
  const dd inv_n(1.0 / (double)p->N);
  const cpx<dd>* twr = static_cast<const cpx<dd>*>(p->tw_row_t);
  const cpx<dd>* twc = static_cast<const cpx<dd>*>(p->tw_col_t);
  const cpx<dd>* por = static_cast<const cpx<dd>*>(p->post_row_t);
  const cpx<dd>* poc = static_cast<const cpx<dd>*>(p->post_col_t);
  m.mark(0);
  rows_forward_stage<dd>(p, false, st, in, Fd, twr, por, p->row_scale, static_cast<const dd*>(p->row_scale_t),
                         nullptr, ov);
  if (p->fused) {
    // column 0 on the side stream: its double-float colatitude transforms
    // bracket the FP64 zonal eliminations; every other column in the fused
    // stage on the main stream, in place in Fd
    m.mark(1);
    const cpx<dd>* pcs = static_cast<const cpx<dd>*>(p->post_col_s_t);
    cudaEventRecord(p->ev_fork, st);
    cudaStreamWaitEvent(p->side, p->ev_fork, 0);
    launch_theta_forward_x<dd>(p, false, p->side, Fd, p->N, 1, p->Kp, p->cols_per_cta, p->col_fft, twc,
                               p->perm_col, pcs, inv_n, 0);
    const int zt = 256;
    sp::launch_zonal_extract(Launch{dim3((p->N + zt - 1) / zt), zt, 0, p->side}, Fd, Z, p->N, p->Kp);
    sp::launch_zonal_scan(false, p->side, Z, p->z_l, p->z_iu, p->z_cu, p->N);
    sp::launch_zonal_insert(Launch{dim3(1), 512, 0, p->side}, Z, Fd, p->N, p->Kp);
    launch_theta_inverse_x<dd>(p, false, p->side, Fd, p->N, 1, p->Kp, p->cols_per_cta, p->col_fft, twc,
                               p->perm_col, poc, inv_n, 0);
    cudaEventRecord(p->ev_join, p->side);
    sp::launch_refine_fused(p->big_col, Launch{dim3(1), p->fuse_threads, p->fuse_smem, st}, Fd, p->N, p->K, p->Kp,
                            p->col_fft, twc, p->perm_col, pcs, poc, p->fc_iu, p->sweeps, p->dev_status);
    m.mark(2);
    m.mark(3);
    cudaStreamWaitEvent(st, p->ev_join, 0);
    m.mark(4);
    rows_inverse_stage<dd>(p, false, st, Fd, out, twr, por, p->row_scale, static_cast<const dd*>(p->row_scale_t),
                           nullptr, ov);
    m.mark(5);
    m.done();
    return;
  }
  m.mark(1);
  launch_theta_forward_x<dd>(p, false, st, Fd, p->N, p->K, p->Kp, p->cols_per_cta, p->col_fft,
                               twc, p->perm_col, static_cast<const cpx<dd>*>(p->post_col_s_t), inv_n, 0);
  cudaEventRecord(p->ev_fork, st);
  cudaStreamWaitEvent(p->side, p->ev_fork, 0);
  {
    const int zt = 256;
    sp::launch_zonal_extract(Launch{dim3((p->N + zt - 1) / zt), zt, 0, p->side}, Fd, Z, p->N, p->Kp);
    sp::launch_zonal_scan(false, p->side, Z, p->z_l, p->z_iu, p->z_cu, p->N);
    sp::launch_zonal_insert(Launch{dim3(1), 512, 0, p->side}, Z, Xd, p->N, p->Kp);
  }
  cudaEventRecord(p->ev_join, p->side);
  m.mark(2);
  for (int s = 0; s <= p->sweeps; ++s)
    sp::launch_refine(solve, Fd, Xd, Y, p->f32_l, p->f32_iu, p->f32_cu, p->N, p->K, p->Kp, s == 0 ? 1 : 0);
  cudaStreamWaitEvent(st, p->ev_join, 0);
  m.mark(3);
  launch_theta_inverse_x<dd>(p, false, st, Xd, p->N, p->K, p->Kp, p->cols_per_cta, p->col_fft,
                               twc, p->perm_col, poc, inv_n, 0);
  m.mark(4);
  rows_inverse_stage<dd>(p, false, st, Xd, out, twr, por, p->row_scale, static_cast<const dd*>(p->row_scale_t),
                         nullptr, ov);
  m.mark(5);
  m.done();
}

// the persistent kernel of the plan's arithmetic; big: with the large-prime passes
cudaError_t batched_occupancy(const sp_plan_s* p, bool big, size_t smem, int* bps) {
  if (p->precision == SP_FP64) return sp::batched_fp64_occupancy(big, kBatchThreadsPerCta, smem, bps);
  return sp::batched_refine_occupancy(big, kBatchThreadsPerCta, smem, bps);
}
void launch_batched_kernel(const sp_plan_s* p, bool big, dim3 grid, size_t smem, cudaStream_t st,
                           const sp::BatchArgs& a) {
  if (p->precision == SP_FP64) sp::launch_batched_fp64(big, grid, kBatchThreadsPerCta, smem, st, a);
  else sp::launch_batched_refine(big, grid, kBatchThreadsPerCta, smem, st, a);
}

int launch_batched(sp_plan_t p, const double* in, double* out, void* workspace, cudaStream_t st) {
  if (p->count == 0) return SP_OK;
  sp::BatchArgs a = p->bargs;
  a.f = in;
  a.u = out;
  a.scratch = static_cast<cpx<double>*>(workspace);
  int* counters = reinterpret_cast<int*>(static_cast<char*>(workspace) + p->off_counter);
  cudaError_t e = cudaMemsetAsync(counters, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(batch counters)");
  StageMarks m{p, st, !p->prof_events.empty() && p->prof_count < p->prof_max};
  m.mark(0);
  const int first[2] = {0, p->bsplit}, n[2] = {p->bsplit, p->count - p->bsplit};
  for (int g = 0; g < 2; ++g) {
    if (n[g] == 0) continue;
    sp::BatchArgs ag = a;
    ag.order = a.order + first[g];
    ag.count = n[g];
    ag.counter = counters + g;
    launch_batched_kernel(p, g == 1, dim3(p->bgrid_g[g]), p->bsmem_g[g], st, ag);
  }
  for (int s = 1; s <= kStages; ++s) m.mark(s);
  m.done();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "batched launch");
  return SP_OK;
}

template <bool ADJ>
int launch_solve(sp_plan_t p, const double* in, double* out, void* workspace, cudaStream_t st) {
  if (p->batched) {
    if (ADJ) return SP_ERR_UNSUPPORTED;
    return launch_batched(p, in, out, workspace, st);
  }
  if (p->precision == SP_FP64) {
    enqueue_fp64(p, ADJ, in, out, workspace, st);
  } else if (p->precision == SP_FP32) {
    enqueue_fp32(p, ADJ, in, out, workspace, st);
  } else {
    if (ADJ) return SP_ERR_UNSUPPORTED;
    enqueue_refine(p, in, out, workspace, st);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "solve launch");
  return SP_OK;
}

std::mutex g_attr_mutex;
bool g_attr_done[64] = {};

// raise the dynamic shared-memory cap of every transform kernel once per
// device to the device maximum, so plans of any size can share the kernels
cudaError_t allow_all_smem(int device) {
  std::lock_guard<std::mutex> lock(g_attr_mutex);
  if (device >= 0 && device < 64 && g_attr_done[device]) return cudaSuccess;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  if (e != cudaSuccess) return e;
  optin -= 1024;  // headroom for the kernels' static shared memory
  cudaError_t r = cudaSuccess;
  auto upd = [&](cudaError_t x) { if (r == cudaSuccess) r = x; };
  upd(sp::allow_transform_smem<double>(optin));
  upd(sp::allow_transform_smem<float>(optin));
  upd(sp::allow_transform_smem<sp::dd>(optin));
  if (r == cudaSuccess && device >= 0 && device < 64) g_attr_done[device] = true;
  return r;
}

bool set_fused_tile(sp_plan_t p, int cols, int threads) {
  // FP32: cols > 0: two buffers, cols columns per CTA; cols < 0: one buffer,
  // -cols columns per CTA; cols = 0: the cluster form (one column per CTA, four
  // CTAs per cluster).  FP32 + refinement: one column per CTA (cols ignored).
  if (p->batched || p->precision == SP_FP64 || threads < 64) return false;
  if (p->precision == SP_FP32_REFINE) {
    const size_t smem = sp::refine_fused_smem(p->N, threads);
    if (smem > 220 * 1024) return false;
    p->fuse_cols = 1;
    p->fuse_threads = threads;
    p->fuse_smem = smem;
    return true;
  }
  const size_t smem = sp::theta_fused_smem(p->N, cols, threads);
  if (smem > 220 * 1024 || 2 * std::max(std::abs(cols), 1) * 32 > threads) return false;
  p->fuse_cols = cols;
  p->fuse_threads = threads;
  p->fuse_smem = smem;
  return true;
}

template <typename S>
void upload_table(const std::vector<cpx<double>>& src, std::vector<char>& dst);

template <>
void upload_table<float>(const std::vector<cpx<double>>& src, std::vector<char>& dst) {
  dst.resize(src.size() * sizeof(cpx<float>));
  cpx<float>* o = reinterpret_cast<cpx<float>*>(dst.data());
  for (size_t i = 0; i < src.size(); ++i) o[i] = {(float)src[i].re, (float)src[i].im};
}

template <>
void upload_table<sp::dd>(const std::vector<cpx<double>>& src, std::vector<char>& dst) {
  dst.resize(src.size() * sizeof(cpx<sp::dd>));
  cpx<sp::dd>* o = reinterpret_cast<cpx<sp::dd>*>(dst.data());
  for (size_t i = 0; i < src.size(); ++i) o[i] = {sp::dd(src[i].re), sp::dd(src[i].im)};
}

void destroy_plan(sp_plan_s* p) {
  for (cudaEvent_t e : p->prof_events) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ov_events) cudaEventDestroy(e);
  if (p->copy) cudaStreamDestroy(p->copy);
  if (p->alt) cudaStreamDestroy(p->alt);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->dev) cudaFree(p->dev);
  p->magic = 0;
  delete p;
}

}  // namespace

namespace {
int tune_single(sp_plan_t p);  // defined with the batched tuner
}  // namespace

extern "C" {

int sphere_poisson_plan(sp_plan_t* plan, int n_theta, int n_lambda, int precision,
                        int refine_sweeps, unsigned flags, size_t* workspace_bytes) {
  if (!plan) return SP_ERR_NULL;
  *plan = nullptr;
  if (n_theta < 1 || n_lambda < 2 || (n_lambda & 1)) return SP_ERR_BAD_SIZE;
  if (n_theta > kMaxLen || n_lambda / 2 > kMaxLen) return SP_ERR_BAD_SIZE;
  if (precision != SP_FP64 && precision != SP_FP32 && precision != SP_FP32_REFINE) return SP_ERR_UNSUPPORTED;
  if ((flags & ~(SP_FLAG_AUTOTUNE | SP_FLAG_POLES)) != 0 || refine_sweeps < 0 || refine_sweeps > 16)
    return SP_ERR_BAD_ARG;
  const bool poles = (flags & SP_FLAG_POLES) != 0;
  if (poles && precision != SP_FP64) return SP_ERR_UNSUPPORTED;
  if (poles && 2 * n_theta > kMaxLen) return SP_ERR_BAD_SIZE;

  FftDesc rd, cd, pd{};
  if (!make_fft_desc(n_lambda / 2, &rd) || !make_fft_desc(n_theta, &cd)) return SP_ERR_BAD_SIZE;
  if (poles && !make_fft_desc(2 * n_theta, &pd)) return SP_ERR_BAD_SIZE;

  sp_plan_s* p = new (std::nothrow) sp_plan_s();
  if (!p) return SP_ERR_CUDA;
  p->poles = poles;
  p->nt = poles ? n_theta + 1 : n_theta;
  p->nl = n_lambda;
  p->L = n_lambda / 2;
  p->N = n_theta;
  p->K = p->L + 1;
  p->Kp = (p->K + 1) & ~1;
  p->precision = precision;
  p->sweeps = precision == SP_FP32_REFINE ? refine_sweeps : 0;
  p->row_fft = rd;
  p->col_fft = cd;
  p->big_row = needs_big(rd);
  p->big_col = needs_big(cd);
  const size_t csz = esize(precision);
  // tiles: rows per CTA and columns per CTA, powers of two up to 8 within the budget
  p->rows_per_cta = 1;
  while (p->rows_per_cta < 8 && (size_t)(2 * p->rows_per_cta) * p->L * csz <= 96 * 1024 &&
         2 * p->rows_per_cta <= p->nt)
    p->rows_per_cta *= 2;
  p->cols_per_cta = 1;
  while (p->cols_per_cta < 8 && (size_t)(2 * p->cols_per_cta) * p->N * csz <= kSmemBudget &&
         2 * p->cols_per_cta <= p->Kp)
    p->cols_per_cta *= 2;
  p->row_smem = (size_t)p->rows_per_cta * p->L * csz;
  p->col_smem = (size_t)p->cols_per_cta * p->N * csz;
  p->row_threads = fft_threads(rd, p->rows_per_cta);
  p->col_threads = fft_threads(cd, p->cols_per_cta);
  p->zcol_threads = fft_threads(cd, 1);
  p->zcol_smem = (size_t)p->N * sizeof(cpx<double>);
  if (poles) {
    p->pole_fft = pd;
    p->big_pole = needs_big(pd);
    p->pole_threads = fft_threads(pd, 1);
    p->pole_smem = (size_t)pd.L * sizeof(cpx<double>);
  }
  if (p->row_threads < 0 || p->col_threads < 0 || p->row_smem > 220 * 1024 || p->col_smem > 220 * 1024 ||
      p->zcol_smem > 220 * 1024 || p->pole_threads < 0 || p->pole_smem > 220 * 1024) {
    delete p;
    return SP_ERR_BAD_SIZE;
  }
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t grid = (size_t)p->N * p->Kp;
  const size_t zbytes = (size_t)p->N * 2 * sizeof(cpx<double>);
  if (precision == SP_FP64) {
    p->ws_bytes = (size_t)std::max(p->nt, p->N) * p->Kp * sizeof(cpx<double>);   // poles: N + 1 sample rows
  } else if (precision == SP_FP32) {
    p->off_z = align(grid * sizeof(cpx<float>));
    p->ws_bytes = p->off_z + zbytes;
  } else {
    p->off_x = align(grid * sizeof(cpx<sp::dd>));
    p->off_y = p->off_x + align(grid * sizeof(cpx<sp::dd>));
    p->off_z = p->off_y + align(grid * sizeof(cpx<float>));
    p->ws_bytes = p->off_z + zbytes;
  }

  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return cuda_fail(cudaGetLastError(), "cudaGetDevice");
  }
  if (cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
    delete p;
    return cuda_fail(cudaGetLastError(), "cudaDeviceGetAttribute");
  }

  // host tables
  const size_t cd_sz = sizeof(cpx<double>);
  std::vector<cpx<double>> tw_row = stage_twiddles(rd), tw_col = stage_twiddles(cd);
  std::vector<cpx<double>> post_row(p->L + 1), post_col(p->N + 1);
  for (int k = 0; k <= p->L; ++k) unit_root(k, n_lambda, &post_row[k].re, &post_row[k].im);
  for (int j = 0; j <= p->N; ++j) unit_root(j, 4L * p->N, &post_col[j].re, &post_col[j].im);
  std::vector<cpx<double>> post_col_s(p->N + 1);
  for (int j = 0; j <= p->N; ++j) post_col_s[j] = {post_col[j].re * (0.5 / p->N), post_col[j].im * (0.5 / p->N)};
  std::vector<int> perm_row, perm_col;
  digit_reversal(rd, perm_row);
  digit_reversal(cd, perm_col);
  // exp(-i theta_i) with theta_i = 2 pi (2i + 1) / (4N) (pole-free) or 2 pi (2i) / (4N) (poles), exactly reduced
  auto theta_root = [&](int i, double* re, double* im) { unit_root(poles ? 2L * i : 2L * i + 1, 4L * p->N, re, im); };
  std::vector<double> row_scale(p->nt);
  for (int i = 0; i < p->nt; ++i) {
    double re, im;
    theta_root(i, &re, &im);  // sin(theta_i) = -im (exactly 0 at the poles)
    row_scale[i] = (im * im) / (double)n_lambda;
  }
  std::vector<cpx<double>> tw_pole;
  std::vector<int> perm_pole;
  if (poles) {
    tw_pole = stage_twiddles(pd);
    digit_reversal(pd, perm_pole);
  }
  std::vector<char> t_tw_row, t_tw_col, t_post_row, t_post_col, t_post_col_s, t_scale;
  if (precision == SP_FP32) {
    t_scale.resize(p->nt * sizeof(float));
    for (int i = 0; i < p->nt; ++i) reinterpret_cast<float*>(t_scale.data())[i] = (float)row_scale[i];
    upload_table<float>(tw_row, t_tw_row);
    upload_table<float>(tw_col, t_tw_col);
    upload_table<float>(post_row, t_post_row);
    upload_table<float>(post_col, t_post_col);
    upload_table<float>(post_col_s, t_post_col_s);
  } else if (precision == SP_FP32_REFINE) {
    t_scale.resize(p->nt * sizeof(sp::dd));
    for (int i = 0; i < p->nt; ++i) reinterpret_cast<sp::dd*>(t_scale.data())[i] = sp::dd(row_scale[i]);
    upload_table<sp::dd>(tw_row, t_tw_row);
    upload_table<sp::dd>(tw_col, t_tw_col);
    upload_table<sp::dd>(post_row, t_post_row);
    upload_table<sp::dd>(post_col, t_post_col);
    upload_table<sp::dd>(post_col_s, t_post_col_s);
  }

  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align(off + bytes);
    return o;
  };
  size_t o_tw_row = take(tw_row.size() * cd_sz), o_tw_col = take(tw_col.size() * cd_sz);
  size_t o_post_row = take((p->L + 1) * cd_sz), o_post_col = take((p->N + 1) * cd_sz);
  size_t o_post_col_s = take((p->N + 1) * cd_sz);
  size_t o_scale = take(p->nt * sizeof(double));
  size_t o_plain = take(p->nt * sizeof(double));
  size_t o_sin2 = take(p->nt * sizeof(double));
  size_t o_geo = take((size_t)(2 * p->nt + 2 * p->nl) * sizeof(double));
  size_t o_mean_w = take(p->nt * sizeof(double));
  size_t o_perm_row = take(p->L * sizeof(int)), o_perm_col = take(p->N * sizeof(int));
  size_t o_tw_pole = take(tw_pole.size() * cd_sz), o_perm_pole = take(perm_pole.size() * sizeof(int));
  size_t o_status = take(sizeof(int));
  size_t o_t_tw_row = take(t_tw_row.size()), o_t_tw_col = take(t_tw_col.size());
  size_t o_t_post_row = take(t_post_row.size()), o_t_post_col = take(t_post_col.size());
  size_t o_t_scale = take(t_scale.size());
  size_t o_t_post_col_s = take(t_post_col_s.size());
  const size_t fac64 = precision == SP_FP64 ? grid * sizeof(double) : 0;
  const size_t fac32 = precision == SP_FP64 ? 0 : grid * sizeof(float);
  const size_t facz = precision == SP_FP64 ? 0 : (size_t)p->N * 2 * sizeof(double);
  const size_t faccol = precision != SP_FP64 ? (size_t)p->K * p->N * sizeof(float) : 0;
  const size_t o_fac_begin = off;
  size_t o_l = take(fac64), o_iu = take(fac64), o_cu = take(fac64);
  size_t o_l32 = take(fac32), o_iu32 = take(fac32), o_cu32 = take(fac32);
  size_t o_zl = take(facz), o_ziu = take(facz), o_zcu = take(facz);
  size_t o_fciu = take(faccol);
  const size_t total = off;

  int rc = SP_OK;
  auto step = [&](cudaError_t err, const char* what) {
    if (rc == SP_OK && err != cudaSuccess) rc = cuda_fail(err, what);
  };
  step(cudaMalloc(&p->dev, total), "cudaMalloc(plan tables)");
  if (rc != SP_OK) {
    p->dev = nullptr;
    destroy_plan(p);
    return rc;
  }
  char* base = static_cast<char*>(p->dev);
  p->tw_row = reinterpret_cast<cpx<double>*>(base + o_tw_row);
  p->tw_col = reinterpret_cast<cpx<double>*>(base + o_tw_col);
  p->post_row = reinterpret_cast<cpx<double>*>(base + o_post_row);
  p->post_col = reinterpret_cast<cpx<double>*>(base + o_post_col);
  p->post_col_s = reinterpret_cast<cpx<double>*>(base + o_post_col_s);
  p->row_scale = reinterpret_cast<double*>(base + o_scale);
  p->row_plain = reinterpret_cast<double*>(base + o_plain);
  p->sin2 = reinterpret_cast<double*>(base + o_sin2);
  p->geo = reinterpret_cast<double*>(base + o_geo);
  p->mean_w = reinterpret_cast<double*>(base + o_mean_w);
  p->perm_row = reinterpret_cast<int*>(base + o_perm_row);
  p->perm_col = reinterpret_cast<int*>(base + o_perm_col);
  p->tw_pole = poles ? reinterpret_cast<cpx<double>*>(base + o_tw_pole) : nullptr;
  p->perm_pole = poles ? reinterpret_cast<int*>(base + o_perm_pole) : nullptr;
  p->dev_status = reinterpret_cast<int*>(base + o_status);
  p->tw_row_t = base + o_t_tw_row;
  p->tw_col_t = base + o_t_tw_col;
  p->post_row_t = base + o_t_post_row;
  p->post_col_t = base + o_t_post_col;
  p->row_scale_t = base + o_t_scale;
  p->post_col_s_t = base + o_t_post_col_s;
  p->fac_l = reinterpret_cast<double*>(base + o_l);
  p->fac_iu = reinterpret_cast<double*>(base + o_iu);
  p->fac_cu = reinterpret_cast<double*>(base + o_cu);
  p->f32_l = reinterpret_cast<float*>(base + o_l32);
  p->f32_iu = reinterpret_cast<float*>(base + o_iu32);
  p->f32_cu = reinterpret_cast<float*>(base + o_cu32);
  p->z_l = reinterpret_cast<double*>(base + o_zl);
  p->z_iu = reinterpret_cast<double*>(base + o_ziu);
  p->z_cu = reinterpret_cast<double*>(base + o_zcu);
  p->fc_iu = reinterpret_cast<float*>(base + o_fciu);
  p->magic = kMagic;

  auto up = [&](void* dst, const void* src, size_t bytes, const char* what) {
    if (bytes) step(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice), what);
  };
  up(p->tw_row, tw_row.data(), tw_row.size() * cd_sz, "copy tw_row");
  up(p->tw_col, tw_col.data(), tw_col.size() * cd_sz, "copy tw_col");
  up(p->post_row, post_row.data(), (p->L + 1) * cd_sz, "copy post_row");
  up(p->post_col, post_col.data(), (p->N + 1) * cd_sz, "copy post_col");
  up(p->post_col_s, post_col_s.data(), (p->N + 1) * cd_sz, "copy post_col_s");
  up(p->post_col_s_t, t_post_col_s.data(), t_post_col_s.size(), "copy post_col_s_t");
  up(p->row_scale, row_scale.data(), p->nt * sizeof(double), "copy row_scale");
  {
    std::vector<double> plain(p->nt, 1.0 / (double)n_lambda);
    up(p->row_plain, plain.data(), p->nt * sizeof(double), "copy row_plain");
    std::vector<double> s2(p->nt);
    for (int i = 0; i < p->nt; ++i) {
      double re, im;
      theta_root(i, &re, &im);  // sin(theta_i) = -im
      s2[i] = im * im;
    }
    up(p->sin2, s2.data(), p->nt * sizeof(double), "copy sin2");
    // theta_i = 2 pi (2i + 1) / (4N), lambda_q = 2 pi q / n - pi
    std::vector<double> geo(2 * p->nt + 2 * p->nl);
    for (int i = 0; i < p->nt; ++i) {
      double re, im;
      theta_root(i, &re, &im);
      geo[i] = -im;
      geo[p->nt + i] = re;
    }
    for (int q = 0; q < p->nl; ++q) {
      double re, im;
      unit_root(q, p->nl, &re, &im);
      geo[2 * p->nt + q] = -re;
      geo[2 * p->nt + p->nl + q] = im;
    }
    up(p->geo, geo.data(), geo.size() * sizeof(double), "copy geo");
    // row weights of the mean of f: the w-quadrature of eq. integrationCoeffs on
    // the colatitude coefficients of the lambda mean (the theta-Nyquist mode
    // dropped), divided by 4 pi and written on the samples:
    //   mean = sum_i w_i fbar_i,  w_i = (2/m) (1 + 2 sum_{j even, 2 <= j <= N-1} cos(j theta_i) / (1 - j^2)),
    // with j theta_i = 2 pi j (2i + 1) / (4N) reduced exactly through a table of cos(2 pi r / 4N)
    const long M4 = 4L * p->N;
    std::vector<double> c4(M4);
    for (long r = 0; r < M4; ++r) {
      double re, im;
      unit_root(r, M4, &re, &im);
      c4[r] = re;
    }
    // On the grid with poles j theta_i = 2 pi j (2i) / (4N), and the doubled
    // grid holds the interior rows twice but each pole once: the pole rows'
    // weights are halved.
    std::vector<double> mw(p->nt);
    for (int i = 0; i < p->nt; ++i) {
      const long step = (2L * (poles ? 2L * i : 2L * i + 1)) % M4;
      long r = 0;
      double sum = 0.0;
      for (int j = 2; j <= p->N - 1; j += 2) {
        r += step;
        if (r >= M4) r -= M4;
        sum += c4[r] / (1.0 - (double)j * (double)j);
      }
      const double half = (poles && (i == 0 || i == p->N)) ? 0.5 : 1.0;
      mw[i] = half * (1.0 + 2.0 * sum) / (double)p->N / (double)n_lambda;
    }
    up(p->mean_w, mw.data(), p->nt * sizeof(double), "copy mean_w");
  }
  up(p->perm_row, perm_row.data(), p->L * sizeof(int), "copy perm_row");
  up(p->perm_col, perm_col.data(), p->N * sizeof(int), "copy perm_col");
  if (poles) {
    up(p->tw_pole, tw_pole.data(), tw_pole.size() * cd_sz, "copy tw_pole");
    up(p->perm_pole, perm_pole.data(), perm_pole.size() * sizeof(int), "copy perm_pole");
  }
  up(p->tw_row_t, t_tw_row.data(), t_tw_row.size(), "copy tw_row_t");
  up(p->tw_col_t, t_tw_col.data(), t_tw_col.size(), "copy tw_col_t");
  up(p->post_row_t, t_post_row.data(), t_post_row.size(), "copy post_row_t");
  up(p->post_col_t, t_post_col.data(), t_post_col.size(), "copy post_col_t");
  up(p->row_scale_t, t_scale.data(), t_scale.size(), "copy row_scale_t");
  step(cudaMemset(base + o_fac_begin, 0, total - o_fac_begin), "clear factors");
  step(cudaMemset(p->dev_status, 0, sizeof(int)), "clear status");
  if (rc == SP_OK) {
    int threads = 128, blocks = (2 * p->K + threads - 1) / threads;
    if (precision == SP_FP64) {
      sp::launch_factor<double>(sp::Launch{dim3(blocks), threads, 0, 0}, p->fac_l, p->fac_iu, p->fac_cu, p->N,
                                p->K, p->Kp, true);
    } else {
      // twisted, for k_solve (FP32) and k_refine (FP32 + refinement)
      sp::launch_factor<float>(sp::Launch{dim3(blocks), threads, 0, 0}, p->f32_l, p->f32_iu, p->f32_cu, p->N,
                               p->K, p->Kp, true);
      sp::launch_factor<double>(sp::Launch{dim3(1), threads, 0, 0}, p->z_l, p->z_iu, p->z_cu, p->N, 1, 2, false);
      // per-column pivots of the fused colatitude stages
      sp::launch_factor_cols(sp::Launch{dim3(blocks), threads, 0, 0}, p->fc_iu, p->N, p->K);
    }
    step(cudaGetLastError(), "k_factor launch");
    step(cudaDeviceSynchronize(), "k_factor");
  }
  if (precision != SP_FP64 && rc == SP_OK) {
    // the zonal side path is a chain of one-CTA kernels: at the highest priority
    // they are dispatched ahead of the main stream's queued CTAs instead of
    // waiting for shared memory to free up at the end of a full-grid kernel
    int lo_prio = 0, hi_prio = 0;
    step(cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio), "cudaDeviceGetStreamPriorityRange");
    step(cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, hi_prio), "cudaStreamCreate(side)");
    step(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
    step(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming), "cudaEventCreate");
  }
  step(allow_all_smem(p->device), "shared memory attribute");
  p->pipe_rows = p->pipe_cols = true;
  step(configure_pipes(p), "pipelined kernels");
  // the FP32 form fuses its colatitude stages: one column per CTA, the widest
  // thread count the kernel allows (the tuner may choose otherwise)
  if (precision == SP_FP32)
    p->fused = set_fused_tile(p, p->Kp >= 2 ? -2 : -1, p->big_col ? 256 : 512) ||
               set_fused_tile(p, -1, p->big_col ? 256 : 512);
  else if (precision == SP_FP32_REFINE)
    p->fused = set_fused_tile(p, 1, p->big_col ? 256 : 512) || set_fused_tile(p, 1, 256);
  if (rc == SP_OK && (flags & SP_FLAG_AUTOTUNE)) rc = tune_single(p);
  if (rc != SP_OK) {
    destroy_plan(p);
    return rc;
  }
  if (workspace_bytes) *workspace_bytes = p->ws_bytes;
  *plan = p;
  return SP_OK;
}

}  // extern "C"

namespace {

constexpr int kBatchThreads = kBatchThreadsPerCta;

// host copy of the per-size tables of a batched plan
struct HostClass {
  int nt, nl;
  FftDesc rd, cd;
  std::vector<cpx<double>> tw_row, tw_col, post_row, post_col, post_col_s;
  std::vector<int> perm_row, perm_col;
  std::vector<double> row_scale;
};

void default_tiles(sp::BatchClass& c) {
  const size_t cs = sizeof(cpx<double>), budget = 96 * 1024;
  c.rows = 1;
  while (c.rows < 8 && (size_t)(2 * c.rows) * c.L * cs <= budget && 2 * c.rows <= c.nt) c.rows *= 2;
  c.cols = 1;
  while (c.cols < 8 && (size_t)(2 * c.cols) * c.N * cs <= budget && 2 * c.cols <= c.Kp) c.cols *= 2;
}

size_t class_smem(const sp::BatchClass& c) {
  const size_t cs = sizeof(cpx<double>);
  return std::max((size_t)c.rows * c.L * cs, (size_t)c.cols * c.N * cs);
}

std::string tune_key(const char* gpu, int nt, int nl, int precision) {
  std::ostringstream o;
  o << gpu << "|" << nt << "x" << nl << (precision == SP_FP64 ? "|fp64" : "|fp32_refine");
  std::string k = o.str();
  for (char& ch : k)
    if (ch == ' ') ch = '_';
  return k;
}

// tune cache: one entry per line, a key without spaces followed by numbers
std::map<std::string, std::vector<double>> read_tune_lines(const char* path) {
  std::map<std::string, std::vector<double>> m;
  if (!path) return m;
  std::ifstream in(path);
  std::string line;
  while (std::getline(in, line)) {
    std::istringstream ls(line);
    std::string key;
    if (!(ls >> key)) continue;
    std::vector<double> v;
    double x;
    while (ls >> x) v.push_back(x);
    m[key] = v;
  }
  return m;
}

std::map<std::string, std::pair<int, int>> read_tune_cache(const char* path) {
  std::map<std::string, std::pair<int, int>> m;
  for (auto& kv : read_tune_lines(path))
    if (kv.second.size() >= 2) m[kv.first] = {(int)kv.second[0], (int)kv.second[1]};
  return m;
}

std::string spaceless(std::string k) {
  for (char& ch : k)
    if (ch == ' ') ch = '_';
  return k;
}

const char* precision_tag(int precision) {
  return precision == SP_FP64 ? "fp64" : precision == SP_FP32 ? "fp32" : "fp32_refine";
}

// Plan-time tile tuning of a single plan: the candidate (rows per CTA, threads)
// of the longitude kernels, then (columns per CTA, threads) of the colatitude
// kernels, each timed as whole solves on zero input (fastest of three after a
// warm-up); the fastest is kept and cached per GPU, grid and arithmetic in the
// file named by SPHERE_POISSON_TUNE_CACHE.
int tune_single(sp_plan_t p) {
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, p->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  std::ostringstream ko;
  ko << prop.name << "|" << p->nt << "x" << p->nl << "|single|" << precision_tag(p->precision) << "|"
     << p->sweeps << (p->poles ? "|poles" : "");
  const std::string key = spaceless(ko.str());
  const char* cache_path = std::getenv("SPHERE_POISSON_TUNE_CACHE");
  const size_t csz = esize(p->precision);
  auto set_rows = [&](int r, int t, bool pipe) {
    p->rows_per_cta = r;
    p->row_threads = t;
    p->row_smem = (size_t)r * p->L * csz;
    p->pipe_rows = pipe;
    configure_pipes(p);
  };
  auto set_cols = [&](int q, int t, bool pipe) {
    p->cols_per_cta = q;
    p->col_threads = t;
    p->col_smem = (size_t)q * p->N * csz;
    p->pipe_cols = pipe;
    configure_pipes(p);
  };
  {
    auto cache = read_tune_lines(cache_path);
    auto it = cache.find(key);
    if (it != cache.end() && it->second.size() >= 7) {
      const std::vector<double>& v = it->second;
      set_rows((int)v[0], (int)v[1], v[4] != 0.0);
      set_cols((int)v[2], (int)v[3], v[5] != 0.0);
      if (v.size() >= 10 && p->precision != SP_FP64)
        p->fused = v[7] != 0.0 && set_fused_tile(p, (int)v[8], (int)v[9]);
      return SP_OK;
    }
  }
  const size_t grid_vals = (size_t)p->nt * p->nl;
  double* f = nullptr;
  double* u = nullptr;
  void* ws = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SP_OK;
  auto step = [&](cudaError_t err, const char* what) {
    if (rc == SP_OK && err != cudaSuccess) rc = cuda_fail(err, what);
  };
  step(cudaMalloc(&f, grid_vals * sizeof(double)), "tune buffers");
  step(cudaMalloc(&u, grid_vals * sizeof(double)), "tune buffers");
  step(cudaMalloc(&ws, p->ws_bytes), "tune buffers");
  step(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "tune stream");
  step(cudaEventCreate(&e0), "tune events");
  step(cudaEventCreate(&e1), "tune events");
  if (rc == SP_OK) step(cudaMemset(f, 0, grid_vals * sizeof(double)), "tune buffers");
  auto time_solve = [&]() -> double {
    double best = 1e30;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(e0, st);
      int r = launch_solve<false>(p, f, u, ws, st);
      cudaEventRecord(e1, st);
      if (r != SP_OK || cudaEventSynchronize(e1) != cudaSuccess) {
        cudaGetLastError();
        return 1e30;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, (double)ms);
    }
    return best;
  };
  const int cap_r = p->big_row ? 256 : 512, cap_c = p->big_col ? 256 : 512;
  double best_ms = 1e30;
  // the transform tiles are tuned on the unfused path, then the fused stage's tiles
  const bool fused0 = p->fused;
  const int fc0 = p->fuse_cols, ft0 = p->fuse_threads;
  p->fused = false;
  if (rc == SP_OK) {
    int br = p->rows_per_cta, bt = p->row_threads;
    bool bp = p->pipe_rows;
    best_ms = time_solve();
    for (int r = 1; r <= 8 && r <= p->nt; r *= 2)
      for (int t = 64; t <= cap_r; t *= 2)
        for (int pipe = 0; pipe < 2; ++pipe) {
          if ((size_t)r * p->L * csz > 220 * 1024) continue;
          set_rows(r, t, pipe != 0);
          if (pipe && !p->pipe[0] && !p->pipe[3]) continue;   // the pipelined kernels do not fit
          const double ms = time_solve();
          if (ms < best_ms) {
            best_ms = ms;
            br = r;
            bt = t;
            bp = pipe != 0;
          }
        }
    set_rows(br, bt, bp);
    int bq = p->cols_per_cta, bct = p->col_threads;
    bool bcp = p->pipe_cols;
    for (int q = 1; q <= 8 && q <= p->Kp; q *= 2)
      for (int t = 64; t <= cap_c; t *= 2)
        for (int pipe = 0; pipe < 2; ++pipe) {
          if ((size_t)q * p->N * csz > 220 * 1024) continue;
          set_cols(q, t, pipe != 0);
          if (pipe && !p->pipe[1] && !p->pipe[2]) continue;
          const double ms = time_solve();
          if (ms < best_ms) {
            best_ms = ms;
            bq = q;
            bct = t;
            bcp = pipe != 0;
          }
        }
    set_cols(bq, bct, bcp);
    if (fused0) {
      bool bf = false;
      int bfc = fc0, bft = ft0;
      const std::vector<int> tiles = p->precision == SP_FP32 ? std::vector<int>{-1, -2, -4, 0, 1, 2, 4}
                                                             : std::vector<int>{1};
      for (int q : tiles)
        for (int t = 128; t <= cap_c; t *= 2) {
          if (std::abs(q) > p->Kp) continue;
          if (!set_fused_tile(p, q, t)) continue;
          p->fused = true;
          const double ms = time_solve();
          p->fused = false;
          if (ms < best_ms) {
            best_ms = ms;
            bf = true;
            bfc = q;
            bft = t;
          }
        }
      p->fused = bf && set_fused_tile(p, bfc, bft);
      if (!p->fused) set_fused_tile(p, fc0, ft0);
    }
  } else {
    p->fused = fused0;
  }
  if (st) cudaStreamSynchronize(st);
  cudaFree(f);
  cudaFree(u);
  cudaFree(ws);
  if (st) cudaStreamDestroy(st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc == SP_OK && cache_path && best_ms < 1e29) {
    std::ofstream out(cache_path, std::ios::app);
    out << key << " " << p->rows_per_cta << " " << p->row_threads << " " << p->cols_per_cta << " "
        << p->col_threads << " " << (int)p->pipe_rows << " " << (int)p->pipe_cols << " " << best_ms << " "
        << (int)p->fused << " " << p->fuse_cols << " " << p->fuse_threads << "\n";
  }
  return rc;
}

// Time candidate tiles of one size class on a batch of `reps_problems` copies
// of that size (zero input), through the same persistent kernel.  Returns the
// best (rows, cols) and its time.
int tune_class(sp_plan_t p, int ci, std::vector<sp::BatchClass>& cls, sp::BatchClass* d_cls,
               double* d_f, cpx<double>* d_scratch, int* d_counter, sp::BatchProblem* d_prob, int* d_order,
               int nprob, std::pair<int, int>* best, double* best_ms) {
  sp::BatchClass& c = cls[ci];
  const size_t cs = sizeof(cpx<double>), cap = 200 * 1024;
  std::vector<sp::BatchProblem> prob(nprob);
  std::vector<int> order(nprob);
  const long long per = (long long)c.nt * c.nl;
  for (int i = 0; i < nprob; ++i) {
    prob[i] = {ci, 0, (long long)i * per};
    order[i] = i;
  }
  cudaMemcpy(d_prob, prob.data(), nprob * sizeof(sp::BatchProblem), cudaMemcpyHostToDevice);
  cudaMemcpy(d_order, order.data(), nprob * sizeof(int), cudaMemcpyHostToDevice);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  *best_ms = 1e30;
  const sp::BatchClass saved = c;
  for (int r = 1; r <= 8 && r <= c.nt; r *= 2) {
    for (int q = 1; q <= 8 && q <= c.Kp; q *= 2) {
      if ((size_t)r * c.L * cs > cap || (size_t)q * c.N * cs > cap) continue;
      c.rows = r;
      c.cols = q;
      cudaMemcpy(d_cls + ci, &c, sizeof(sp::BatchClass), cudaMemcpyHostToDevice);
      const size_t smem = class_smem(c);
      const bool big = needs_big(c.row_fft) || needs_big(c.col_fft);
      int bps = 0;
      if (batched_occupancy(p, big, smem, &bps) != cudaSuccess || bps < 1) continue;
      sp::BatchArgs a = p->bargs;
      a.problems = d_prob;
      a.order = d_order;
      a.count = nprob;
      a.f = d_f;
      a.u = d_f + (size_t)nprob * per;
      a.scratch = d_scratch;
      a.counter = d_counter;
      const int grid = std::min(p->bgrid, nprob);
      double ms_min = 1e30;
      for (int rep = 0; rep < 3; ++rep) {
        cudaMemsetAsync(d_counter, 0, sizeof(int), 0);
        cudaEventRecord(e0, 0);
        launch_batched_kernel(p, big, dim3(grid), smem, 0, a);
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) ms_min = std::min(ms_min, (double)ms);
      }
      if (cudaGetLastError() != cudaSuccess) continue;
      if (ms_min < *best_ms) {
        *best_ms = ms_min;
        *best = {r, q};
      }
    }
  }
  c = saved;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return *best_ms < 1e29 ? SP_OK : SP_ERR_CUDA;
}

}  // namespace

extern "C" {

int sphere_poisson_plan_batched(sp_plan_t* plan, int count, const int* n_theta, const int* n_lambda,
                                int precision, int refine_sweeps, unsigned flags, size_t* workspace_bytes) {
  if (!plan) return SP_ERR_NULL;
  *plan = nullptr;
  if (count < 0) return SP_ERR_BAD_ARG;
  if (count > 0 && (!n_theta || !n_lambda)) return SP_ERR_NULL;
  if (precision != SP_FP64 && precision != SP_FP32_REFINE) return SP_ERR_UNSUPPORTED;
  if ((flags & ~SP_FLAG_AUTOTUNE) != 0 || refine_sweeps < 0 || refine_sweeps > 16) return SP_ERR_BAD_ARG;
  const bool refine = precision == SP_FP32_REFINE;
  // validate sizes and form the size classes
  std::map<std::pair<int, int>, int> cls_of;
  std::vector<HostClass> hcls;
  std::vector<int> prob_cls(count);
  for (int b = 0; b < count; ++b) {
    const int nt = n_theta[b], nl = n_lambda[b];
    if (nt < 1 || nl < 2 || (nl & 1) || nt > kMaxLen || nl / 2 > kMaxLen) return SP_ERR_BAD_SIZE;
    auto it = cls_of.find({nt, nl});
    if (it == cls_of.end()) {
      HostClass h;
      h.nt = nt;
      h.nl = nl;
      if (!make_fft_desc(nl / 2, &h.rd) || !make_fft_desc(nt, &h.cd)) return SP_ERR_BAD_SIZE;
      it = cls_of.emplace(std::make_pair(nt, nl), (int)hcls.size()).first;
      hcls.push_back(std::move(h));
    }
    prob_cls[b] = it->second;
  }
  sp_plan_s* p = new (std::nothrow) sp_plan_s();
  if (!p) return SP_ERR_CUDA;
  p->batched = 1;
  p->count = count;
  p->precision = precision;
  p->sweeps = refine ? refine_sweeps : 0;
  p->nt = p->nl = 0;
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    return cuda_fail(cudaGetLastError(), "cudaGetDevice");
  }
  p->offsets.resize(count + 1);
  p->offsets[0] = 0;
  for (int b = 0; b < count; ++b) p->offsets[b + 1] = p->offsets[b] + (size_t)n_theta[b] * n_lambda[b];
  p->total = p->offsets[count];

  // per-class tables
  const int nc = (int)hcls.size();
  std::vector<sp::BatchClass> cls(nc);
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align(off + bytes);
    return o;
  };
  struct Offs {
    size_t tw_row, tw_col, post_row, post_col, post_col_s, perm_row, perm_col, scale, fl, fiu, fcu;
    size_t d_tw_row, d_tw_col, d_post_row, d_post_col, d_post_col_s, d_scale, l32, iu32, cu32, zl, ziu, zcu;
  };
  std::vector<Offs> co(nc);
  bool big = false;
  size_t max_slot = 0;
  for (int c = 0; c < nc; ++c) {
    HostClass& h = hcls[c];
    sp::BatchClass& b = cls[c];
    b.nt = h.nt;
    b.nl = h.nl;
    b.L = h.nl / 2;
    b.N = h.nt;
    b.K = b.L + 1;
    b.Kp = (b.K + 1) & ~1;
    b.row_fft = h.rd;
    b.col_fft = h.cd;
    big = big || needs_big(h.rd) || needs_big(h.cd);
    default_tiles(b);
    // scratch slot in 16-byte units: the half spectrum (FP64), or F, X and the
    // FP32 correction (FP32 + refinement: 16 + 16 + 8 bytes per element)
    const size_t nkp = (size_t)b.N * b.Kp;
    max_slot = std::max(max_slot, refine ? (5 * nkp + 1) / 2 : nkp);
    h.tw_row = stage_twiddles(h.rd);
    h.tw_col = stage_twiddles(h.cd);
    h.post_row.resize(b.L + 1);
    h.post_col.resize(b.N + 1);
    for (int k = 0; k <= b.L; ++k) unit_root(k, b.nl, &h.post_row[k].re, &h.post_row[k].im);
    for (int j = 0; j <= b.N; ++j) unit_root(j, 4L * b.N, &h.post_col[j].re, &h.post_col[j].im);
    h.post_col_s.resize(b.N + 1);
    for (int j = 0; j <= b.N; ++j) h.post_col_s[j] = {h.post_col[j].re * (0.5 / b.N), h.post_col[j].im * (0.5 / b.N)};
    digit_reversal(h.rd, h.perm_row);
    digit_reversal(h.cd, h.perm_col);
    h.row_scale.resize(b.nt);
    for (int i = 0; i < b.nt; ++i) {
      double re, im;
      unit_root(2 * i + 1, 4L * b.N, &re, &im);
      h.row_scale[i] = (im * im) / (double)b.nl;
    }
    const size_t csz = sizeof(cpx<double>), fac = refine ? 0 : (size_t)b.N * b.Kp * sizeof(double);
    const size_t dsz = refine ? sizeof(cpx<sp::dd>) : 0, f32 = refine ? (size_t)b.N * b.Kp * sizeof(float) : 0;
    const size_t fz = refine ? (size_t)b.N * 2 * sizeof(double) : 0;
    Offs& o = co[c];
    o.tw_row = take(h.tw_row.size() * csz);
    o.tw_col = take(h.tw_col.size() * csz);
    o.post_row = take((b.L + 1) * csz);
    o.post_col = take((b.N + 1) * csz);
    o.post_col_s = take((b.N + 1) * csz);
    o.perm_row = take(b.L * sizeof(int));
    o.perm_col = take(b.N * sizeof(int));
    o.scale = take(b.nt * sizeof(double));
    o.fl = take(fac);
    o.fiu = take(fac);
    o.fcu = take(fac);
    o.d_tw_row = take(h.tw_row.size() * dsz);
    o.d_tw_col = take(h.tw_col.size() * dsz);
    o.d_post_row = take((b.L + 1) * dsz);
    o.d_post_col = take((b.N + 1) * dsz);
    o.d_post_col_s = take((b.N + 1) * dsz);
    o.d_scale = take(refine ? b.nt * sizeof(sp::dd) : 0);
    o.l32 = take(f32);
    o.iu32 = take(f32);
    o.cu32 = take(f32);
    o.zl = take(fz);
    o.ziu = take(fz);
    o.zcu = take(fz);
  }
  const size_t o_cls = take(nc * sizeof(sp::BatchClass) + 1);
  const size_t o_prob = take(count * sizeof(sp::BatchProblem) + 1);
  const size_t o_order = take(count * sizeof(int) + 1);
  const size_t total_dev = off;
  p->bbig = big;
  p->bthreads = kBatchThreads;

  int rc = SP_OK;
  auto step = [&](cudaError_t err, const char* what) {
    if (rc == SP_OK && err != cudaSuccess) rc = cuda_fail(err, what);
  };
  step(cudaMalloc(&p->dev, total_dev), "cudaMalloc(batched plan tables)");
  if (rc != SP_OK) {
    p->dev = nullptr;
    destroy_plan(p);
    return rc;
  }
  p->magic = kMagic;
  char* base = static_cast<char*>(p->dev);
  for (int c = 0; c < nc; ++c) {
    HostClass& h = hcls[c];
    sp::BatchClass& b = cls[c];
    const size_t csz = sizeof(cpx<double>);
    b.tw_row = reinterpret_cast<cpx<double>*>(base + co[c].tw_row);
    b.tw_col = reinterpret_cast<cpx<double>*>(base + co[c].tw_col);
    b.post_row = reinterpret_cast<cpx<double>*>(base + co[c].post_row);
    b.post_col = reinterpret_cast<cpx<double>*>(base + co[c].post_col);
    b.post_col_s = reinterpret_cast<cpx<double>*>(base + co[c].post_col_s);
    b.perm_row = reinterpret_cast<int*>(base + co[c].perm_row);
    b.perm_col = reinterpret_cast<int*>(base + co[c].perm_col);
    b.row_scale = reinterpret_cast<double*>(base + co[c].scale);
    b.fl = reinterpret_cast<double*>(base + co[c].fl);
    b.fiu = reinterpret_cast<double*>(base + co[c].fiu);
    b.fcu = reinterpret_cast<double*>(base + co[c].fcu);
    step(cudaMemcpy((void*)b.tw_row, h.tw_row.data(), h.tw_row.size() * csz, cudaMemcpyHostToDevice), "copy");
    step(cudaMemcpy((void*)b.tw_col, h.tw_col.data(), h.tw_col.size() * csz, cudaMemcpyHostToDevice), "copy");
    step(cudaMemcpy((void*)b.post_row, h.post_row.data(), (b.L + 1) * csz, cudaMemcpyHostToDevice), "copy");
    step(cudaMemcpy((void*)b.post_col, h.post_col.data(), (b.N + 1) * csz, cudaMemcpyHostToDevice), "copy");
    step(cudaMemcpy((void*)b.post_col_s, h.post_col_s.data(), (b.N + 1) * csz, cudaMemcpyHostToDevice), "copy");
    step(cudaMemcpy((void*)b.perm_row, h.perm_row.data(), b.L * sizeof(int), cudaMemcpyHostToDevice), "copy");
    step(cudaMemcpy((void*)b.perm_col, h.perm_col.data(), b.N * sizeof(int), cudaMemcpyHostToDevice), "copy");
    step(cudaMemcpy((void*)b.row_scale, h.row_scale.data(), b.nt * sizeof(double), cudaMemcpyHostToDevice), "copy");
    const int threads = 128, blocks = (2 * b.K + threads - 1) / threads;
    if (!refine) {
      const size_t fac = (size_t)b.N * b.Kp * sizeof(double);
      for (const double* t : {b.fl, b.fiu, b.fcu}) step(cudaMemset((void*)t, 0, fac), "clear factors");
      if (rc == SP_OK) {
        sp::launch_factor<double>(sp::Launch{dim3(blocks), threads, 0, 0}, (double*)b.fl, (double*)b.fiu,
                                  (double*)b.fcu, b.N, b.K, b.Kp, false);
        step(cudaGetLastError(), "k_factor launch");
      }
      b.tw_row_d = b.tw_col_d = b.post_row_d = b.post_col_d = b.post_col_s_d = nullptr;
      b.row_scale_d = nullptr;
      b.fl32 = b.fiu32 = b.fcu32 = nullptr;
      b.zl = b.ziu = b.zcu = nullptr;
      continue;
    }
    b.fl = b.fiu = b.fcu = nullptr;
    b.tw_row_d = reinterpret_cast<cpx<sp::dd>*>(base + co[c].d_tw_row);
    b.tw_col_d = reinterpret_cast<cpx<sp::dd>*>(base + co[c].d_tw_col);
    b.post_row_d = reinterpret_cast<cpx<sp::dd>*>(base + co[c].d_post_row);
    b.post_col_d = reinterpret_cast<cpx<sp::dd>*>(base + co[c].d_post_col);
    b.post_col_s_d = reinterpret_cast<cpx<sp::dd>*>(base + co[c].d_post_col_s);
    b.row_scale_d = reinterpret_cast<sp::dd*>(base + co[c].d_scale);
    b.fl32 = reinterpret_cast<float*>(base + co[c].l32);
    b.fiu32 = reinterpret_cast<float*>(base + co[c].iu32);
    b.fcu32 = reinterpret_cast<float*>(base + co[c].cu32);
    b.zl = reinterpret_cast<double*>(base + co[c].zl);
    b.ziu = reinterpret_cast<double*>(base + co[c].ziu);
    b.zcu = reinterpret_cast<double*>(base + co[c].zcu);
    {
      std::vector<char> t;
      auto put = [&](const void* dst, const std::vector<cpx<double>>& src) {
        upload_table<sp::dd>(src, t);
        step(cudaMemcpy((void*)dst, t.data(), t.size(), cudaMemcpyHostToDevice), "copy");
      };
      put(b.tw_row_d, h.tw_row);
      put(b.tw_col_d, h.tw_col);
      put(b.post_row_d, h.post_row);
      put(b.post_col_d, h.post_col);
      put(b.post_col_s_d, h.post_col_s);
      std::vector<sp::dd> sd(b.nt);
      for (int i = 0; i < b.nt; ++i) sd[i] = sp::dd(h.row_scale[i]);
      step(cudaMemcpy((void*)b.row_scale_d, sd.data(), b.nt * sizeof(sp::dd), cudaMemcpyHostToDevice), "copy");
    }
    const size_t f32 = (size_t)b.N * b.Kp * sizeof(float), fz = (size_t)b.N * 2 * sizeof(double);
    for (const float* t : {b.fl32, b.fiu32, b.fcu32}) step(cudaMemset((void*)t, 0, f32), "clear factors");
    for (const double* t : {b.zl, b.ziu, b.zcu}) step(cudaMemset((void*)t, 0, fz), "clear factors");
    if (rc == SP_OK) {
      sp::launch_factor<float>(sp::Launch{dim3(blocks), threads, 0, 0}, (float*)b.fl32, (float*)b.fiu32,
                               (float*)b.fcu32, b.N, b.K, b.Kp, false);
      sp::launch_factor<double>(sp::Launch{dim3(1), threads, 0, 0}, (double*)b.zl, (double*)b.ziu,
                                (double*)b.zcu, b.N, 1, 2, false);
      step(cudaGetLastError(), "k_factor launch");
    }
  }
  step(cudaDeviceSynchronize(), "batched factors");
  // problems, largest first
  std::vector<sp::BatchProblem> prob(count);
  std::vector<int> order(count);
  for (int b = 0; b < count; ++b) {
    prob[b] = {prob_cls[b], 0, (long long)p->offsets[b]};
    order[b] = b;
  }
  // the small-radix group first, then the large-prime group; largest first in each
  auto cls_big = [&](int c) { return needs_big(cls[c].row_fft) || needs_big(cls[c].col_fft); };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const bool bx = cls_big(prob_cls[x]), by = cls_big(prob_cls[y]);
    if (bx != by) return !bx;
    return (size_t)n_theta[x] * n_lambda[x] > (size_t)n_theta[y] * n_lambda[y];
  });
  p->bsplit = 0;
  for (int b = 0; b < count; ++b) p->bsplit += cls_big(prob_cls[b]) ? 0 : 1;
  sp::BatchClass* d_cls = reinterpret_cast<sp::BatchClass*>(base + o_cls);
  sp::BatchProblem* d_prob = reinterpret_cast<sp::BatchProblem*>(base + o_prob);
  int* d_order = reinterpret_cast<int*>(base + o_order);
  p->bargs.classes = d_cls;
  p->bargs.problems = d_prob;
  p->bargs.order = d_order;
  p->bargs.count = count;
  p->bargs.slot = (long long)max_slot;
  p->bargs.sweeps = p->sweeps;
  // persistent grid: every SM filled to the kernel's occupancy
  int sms = 1;
  step(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device), "SM count");
  size_t smem = 0;
  for (auto& b : cls) smem = std::max(smem, class_smem(b));
  int bps = 0;
  step(batched_occupancy(p, p->bbig, std::max(smem, (size_t)200 * 1024), &bps), "occupancy");
  p->bgrid = std::max(1, std::min(count, sms * std::max(bps, 1)));   // the tuner's timing grid

  // autotuning of the transform tiles per size class
  if (rc == SP_OK && count > 0 && (flags & SP_FLAG_AUTOTUNE)) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, p->device);
    const char* cache_path = std::getenv("SPHERE_POISSON_TUNE_CACHE");
    auto cache = read_tune_cache(cache_path);
    std::vector<std::string> new_lines;
    // scratch for the timing batches: nprob problems of the largest class
    const int nprob = std::max(1, p->bgrid);
    size_t max_vals = 0;
    for (auto& b : cls) max_vals = std::max(max_vals, (size_t)b.nt * b.nl);
    double* d_f = nullptr;
    cpx<double>* d_scr = nullptr;
    int* d_cnt = nullptr;
    sp::BatchProblem* d_tp = nullptr;
    int* d_to = nullptr;
    step(cudaMalloc(&d_f, 2 * (size_t)nprob * max_vals * sizeof(double)), "tune buffers");
    step(cudaMalloc(&d_scr, (size_t)p->bgrid * max_slot * sizeof(cpx<double>)), "tune buffers");
    step(cudaMalloc(&d_cnt, 256), "tune buffers");
    step(cudaMalloc(&d_tp, nprob * sizeof(sp::BatchProblem)), "tune buffers");
    step(cudaMalloc(&d_to, nprob * sizeof(int)), "tune buffers");
    if (rc == SP_OK) {
      step(cudaMemset(d_f, 0, 2 * (size_t)nprob * max_vals * sizeof(double)), "tune buffers");
      step(cudaMemcpy(d_cls, cls.data(), nc * sizeof(sp::BatchClass), cudaMemcpyHostToDevice), "copy classes");
    }
    for (int c = 0; c < nc && rc == SP_OK; ++c) {
      const std::string key = tune_key(prop.name, cls[c].nt, cls[c].nl, p->precision);
      auto it = cache.find(key);
      if (it != cache.end()) {
        cls[c].rows = it->second.first;
        cls[c].cols = it->second.second;
        continue;
      }
      std::pair<int, int> best{cls[c].rows, cls[c].cols};
      double ms = 0;
      if (tune_class(p, c, cls, d_cls, d_f, d_scr, d_cnt, d_tp, d_to, nprob, &best, &ms) == SP_OK) {
        cls[c].rows = best.first;
        cls[c].cols = best.second;
        std::ostringstream o;
        o << key << " " << best.first << " " << best.second << " " << ms;
        new_lines.push_back(o.str());
      }
      step(cudaMemcpy(d_cls + c, &cls[c], sizeof(sp::BatchClass), cudaMemcpyHostToDevice), "copy class");
    }
    cudaFree(d_f);
    cudaFree(d_scr);
    cudaFree(d_cnt);
    cudaFree(d_tp);
    cudaFree(d_to);
    if (cache_path && !new_lines.empty()) {
      std::ofstream out(cache_path, std::ios::app);
      for (auto& l : new_lines) out << l << "\n";
    }
  }
  // per group: shared memory of its largest class, a persistent grid at the
  // kernel's occupancy, at most one CTA per problem
  smem = 0;
  for (auto& b : cls) smem = std::max(smem, class_smem(b));
  p->bsmem = smem;
  step(cudaMemcpy(d_cls, cls.data(), nc * sizeof(sp::BatchClass), cudaMemcpyHostToDevice), "copy classes");
  if (count > 0) {
    step(cudaMemcpy(d_prob, prob.data(), count * sizeof(sp::BatchProblem), cudaMemcpyHostToDevice), "copy problems");
    step(cudaMemcpy(d_order, order.data(), count * sizeof(int), cudaMemcpyHostToDevice), "copy order");
    p->bgrid = 1;
    for (int g = 0; g < 2; ++g) {
      const int n = g == 0 ? p->bsplit : count - p->bsplit;
      size_t gs = 0;
      for (int c = 0; c < nc; ++c)
        if (cls_big(c) == (g == 1)) gs = std::max(gs, class_smem(cls[c]));
      p->bsmem_g[g] = gs;
      p->bgrid_g[g] = 0;
      if (n == 0) continue;
      int gbps = 0;
      step(batched_occupancy(p, g == 1, gs, &gbps), "occupancy");
      p->bgrid_g[g] = std::max(1, std::min(n, sms * std::max(gbps, 1)));
      p->bgrid = std::max(p->bgrid, p->bgrid_g[g]);
    }
  }
  p->off_counter = align((size_t)p->bgrid * max_slot * sizeof(cpx<double>));
  p->ws_bytes = p->off_counter + 256;
  step(allow_all_smem(p->device), "shared memory attribute");
  if (rc != SP_OK) {
    destroy_plan(p);
    return rc;
  }
  if (workspace_bytes) *workspace_bytes = p->ws_bytes;
  *plan = p;
  return SP_OK;
}

int sphere_poisson_batch_offsets(sp_plan_t plan, size_t* offsets) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!offsets) return SP_ERR_NULL;
  if (!plan->batched) {
    offsets[0] = 0;
    offsets[1] = (size_t)plan->nt * plan->nl;
    return SP_OK;
  }
  for (size_t i = 0; i < plan->offsets.size(); ++i) offsets[i] = plan->offsets[i];
  return SP_OK;
}

int sphere_poisson_workspace_size(sp_plan_t plan, size_t* workspace_bytes) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!workspace_bytes) return SP_ERR_NULL;
  *workspace_bytes = plan->ws_bytes;
  return SP_OK;
}

int sphere_poisson_solve(sp_plan_t plan, const double* f, double* u, void* workspace,
                         size_t workspace_bytes, void* stream, double* f_mean_out) {
  int rc = check_arrays(plan, f, u, workspace, workspace_bytes);
  if (rc != SP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (f_mean_out) {
    if (plan->batched) return SP_ERR_UNSUPPORTED;
    if ((uintptr_t)f_mean_out & 7) return SP_ERR_MISALIGNED;
    rc = enqueue_mean(plan, f, workspace, f_mean_out, nullptr, st);  // before the solve reuses the workspace
    if (rc != SP_OK) return rc;
  }
  return launch_solve<false>(plan, f, u, workspace, st);
}

int sphere_poisson_solve_adjoint(sp_plan_t plan, const double* ubar, double* fbar, void* workspace,
                                 size_t workspace_bytes, void* stream) {
  int rc = check_arrays(plan, ubar, fbar, workspace, workspace_bytes);
  if (rc != SP_OK) return rc;
  return launch_solve<true>(plan, ubar, fbar, workspace, static_cast<cudaStream_t>(stream));
}

int sphere_poisson_host_buffer_size(sp_plan_t plan, size_t* device_buffer_bytes) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!device_buffer_bytes) return SP_ERR_NULL;
  const size_t values = plan->batched ? plan->total : (size_t)plan->nt * plan->nl;
  size_t grid = (values * sizeof(double) + 255) & ~(size_t)255;
  *device_buffer_bytes = 2 * grid + plan->ws_bytes;
  return SP_OK;
}

int sphere_poisson_solve_host(sp_plan_t plan, const double* f_host, double* u_host, void* device_buffer,
                              size_t device_buffer_bytes, void* stream, double* f_mean_out) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!f_host || !u_host || !device_buffer) return SP_ERR_NULL;
  if ((uintptr_t)device_buffer & 15) return SP_ERR_MISALIGNED;
  if (f_mean_out && plan->batched) return SP_ERR_UNSUPPORTED;
  size_t need = 0;
  sphere_poisson_host_buffer_size(plan, &need);
  if (device_buffer_bytes < need) return SP_ERR_WORKSPACE;
  int drc = on_plan_device(plan);
  if (drc != SP_OK) return drc;
  const size_t bytes = (plan->batched ? plan->total : (size_t)plan->nt * plan->nl) * sizeof(double);
  const size_t grid = (bytes + 255) & ~(size_t)255;
  char* base = static_cast<char*>(device_buffer);
  double* d_f = reinterpret_cast<double*>(base);
  double* d_u = reinterpret_cast<double*>(base + grid);
  void* ws = base + 2 * grid;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // after the solve, the workspace is free: the mean of f and max |f| go to its
  // slot mean_parts(plan), and the call returns the warning when the mean is not
  // zero to rounding
  double mm[2] = {0.0, 0.0};
  auto mean_check = [&]() -> int {
    const int nparts = mean_parts(plan);
    double2* res = static_cast<double2*>(ws) + nparts;
    int rc = enqueue_mean(plan, d_f, ws, &res->x, &res->y, st);
    if (rc != SP_OK) return rc;
    SP_CUDA(cudaMemcpyAsync(mm, res, sizeof mm, cudaMemcpyDeviceToHost, st));
    return SP_OK;
  };
  auto mean_status = [&]() -> int {
    *f_mean_out = mm[0];
    return std::fabs(mm[0]) > kMeanWarnFactor * mm[1] ? SP_WARN_NONZERO_MEAN : SP_OK;
  };
  if (plan->batched || plan->nt < 2 * kHostChunks) {
    SP_CUDA(cudaMemcpyAsync(d_f, f_host, bytes, cudaMemcpyHostToDevice, st));
    int rc = launch_solve<false>(plan, d_f, d_u, ws, st);
    if (rc != SP_OK) return rc;
    SP_CUDA(cudaMemcpyAsync(u_host, d_u, bytes, cudaMemcpyDeviceToHost, st));
    if (f_mean_out && (rc = mean_check()) != SP_OK) return rc;
    SP_CUDA(cudaStreamSynchronize(st));
    if ((rc = take_device_status(plan, st)) != SP_OK) return rc;
    return f_mean_out ? mean_status() : SP_OK;
  }
  // copies overlapped with the longitude transforms, in kHostChunks row chunks
  if (!plan->copy) {
    SP_CUDA(cudaStreamCreateWithFlags(&plan->copy, cudaStreamNonBlocking));
    SP_CUDA(cudaStreamCreateWithFlags(&plan->alt, cudaStreamNonBlocking));
    plan->ov_events.assign(2 * kHostChunks + 5, nullptr);
    for (cudaEvent_t& e : plan->ov_events) SP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  const HostOverlap ov{f_host, u_host, d_f, d_u, plan->copy, plan->alt, plan->ov_events.data() + 1,
                       plan->ov_events.data() + 1 + kHostChunks, plan->ov_events.data() + 1 + 2 * kHostChunks,
                       kHostChunks};
  SP_CUDA(cudaEventRecord(plan->ov_events[0], st));     // the copies follow earlier work on the stream
  SP_CUDA(cudaStreamWaitEvent(plan->copy, plan->ov_events[0], 0));
  if (plan->precision == SP_FP64) enqueue_fp64(plan, false, d_f, d_u, ws, st, &ov);
  else if (plan->precision == SP_FP32) enqueue_fp32(plan, false, d_f, d_u, ws, st, &ov);
  else enqueue_refine(plan, d_f, d_u, ws, st, &ov);
  SP_CUDA(cudaGetLastError());
  if (f_mean_out) {
    int rc = mean_check();
    if (rc != SP_OK) return rc;
  }
  SP_CUDA(cudaStreamSynchronize(plan->copy));
  SP_CUDA(cudaStreamSynchronize(st));
  const int drc2 = take_device_status(plan, st);
  if (drc2 != SP_OK) return drc2;
  return f_mean_out ? mean_status() : SP_OK;
}

int sphere_poisson_device_status(sp_plan_t plan, void* stream) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  const int drc = on_plan_device(plan);
  if (drc != SP_OK) return drc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SP_CUDA(cudaStreamSynchronize(st));
  return take_device_status(plan, st);
}

int sphere_poisson_wait_selftest(sp_plan_t plan, unsigned polls, void* stream) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!plan->dev_status) return SP_ERR_UNSUPPORTED;
  const int drc = on_plan_device(plan);
  if (drc != SP_OK) return drc;
  sp::launch_wait_selftest(plan->dev_status, polls, static_cast<cudaStream_t>(stream));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SP_OK : cuda_fail(e, "wait self-test launch");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free solve: the workspace is this fixed device array.  Host code
// must not pass the symbol itself to a kernel (on the host it names a host-side
// stand-in); the device address is looked up once per device below.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[SP_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// device address of g_noalloc_scratch on the current device (set up on first use)
int noalloc_scratch(int device, void** ptr) {
  if (device < 0 || device >= kMaxDevices) return SP_ERR_BAD_ARG;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
    if (!p) return SP_ERR_CUDA;
    g_noalloc_ptr[device] = p;
  }
  *ptr = g_noalloc_ptr[device];
  return SP_OK;
}
}  // namespace

extern "C" {

int sphere_poisson_solve_noalloc(sp_plan_t plan, const double* f, double* u, void* stream) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!f || !u) return SP_ERR_NULL;
  if (((uintptr_t)f | (uintptr_t)u) & 15) return SP_ERR_MISALIGNED;
  if (plan->ws_bytes > SP_NOALLOC_SCRATCH_BYTES) return SP_ERR_SCRATCH_LIMIT;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != plan->device) return SP_ERR_BAD_ARG;
  void* scratch = nullptr;
  int rc = noalloc_scratch(dev, &scratch);
  if (rc != SP_OK) return rc;
  return launch_solve<false>(plan, f, u, scratch, static_cast<cudaStream_t>(stream));
}

static int check_transform_plan(sp_plan_t plan, const void* a, const void* b, const void* ws, size_t ws_bytes) {
  int rc = check_arrays(plan, a, b, ws, ws_bytes);
  if (rc != SP_OK) return rc;
  if (plan->batched || plan->precision != SP_FP64 || plan->poles) return SP_ERR_UNSUPPORTED;
  return SP_OK;
}

// forward transforms of f (no sin^2 weight) into W, coefficient sign convention
static void enqueue_coeffs2(sp_plan_t p, const double* f, cpx<double>* W, int kcols, cudaStream_t st) {
  using sp::Launch;
  const int K = kcols;
  launch_rows_forward_x<double>(p, false, st, f, W, p->nt, p->nl, p->Kp, p->rows_per_cta,
                                  p->row_fft, p->tw_row, p->perm_row, p->post_row, p->row_plain, p->row_plain,
                                  nullptr);
  launch_theta_forward_x<double>(p, false, st, W, p->N, K, p->Kp, p->cols_per_cta, p->col_fft,
                                   p->tw_col, p->perm_col, p->post_col_s, 1.0 / p->N, 2);
}

int sphere_poisson_coeffs2(sp_plan_t plan, const double* f, void* coeffs, void* workspace, size_t workspace_bytes,
                           void* stream) {
  int rc = check_transform_plan(plan, f, coeffs, workspace, workspace_bytes);
  if (rc != SP_OK) return rc;
  (void)workspace;
  enqueue_coeffs2(plan, f, static_cast<cpx<double>*>(coeffs), plan->K, static_cast<cudaStream_t>(stream));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SP_OK : cuda_fail(e, "coeffs2 launch");
}

int sphere_poisson_sample(sp_plan_t plan, const void* coeffs, double* f, void* workspace, size_t workspace_bytes,
                          void* stream) {
  int rc = check_transform_plan(plan, coeffs, f, workspace, workspace_bytes);
  if (rc != SP_OK) return rc;
  using sp::Launch;
  sp_plan_t p = plan;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cpx<double>* W = static_cast<cpx<double>*>(workspace);
  cudaError_t e = cudaMemcpyAsync(W, coeffs, (size_t)p->N * p->Kp * sizeof(cpx<double>), cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "sample copy");
  launch_theta_inverse_x<double>(p, false, st, W, p->N, p->K, p->Kp, p->cols_per_cta, p->col_fft,
                                   p->tw_col, p->perm_col, p->post_col, 1.0 / p->N, 2);
  launch_rows_inverse_x<double>(p, false, st, W, f, p->nt, p->nl, p->Kp, p->rows_per_cta,
                                  p->row_fft, p->tw_row, p->perm_row, p->post_row, p->row_scale, p->row_scale,
                                  nullptr);
  e = cudaGetLastError();
  return e == cudaSuccess ? SP_OK : cuda_fail(e, "sample launch");
}

int sphere_poisson_sum2(sp_plan_t plan, const double* f, double* result, void* workspace, size_t workspace_bytes,
                        void* stream) {
  int rc = check_transform_plan(plan, f, result, workspace, workspace_bytes);
  if (rc != SP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cpx<double>* W = static_cast<cpx<double>*>(workspace);
  enqueue_coeffs2(plan, f, W, 1, st);  // only the k = 0 column is transformed in colatitude
  sp::launch_sum2_finish(st, W, plan->N, plan->Kp, result);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SP_OK : cuda_fail(e, "sum2 launch");
}

namespace {
// workspace of the derivative operators: `spectra` half spectra of N x Kp
// complex doubles, then the chunk sums of the division by sin theta
size_t spectrum_bytes(sp_plan_t p) { return ((size_t)p->N * p->Kp * sizeof(cpx<double>) + 255) & ~(size_t)255; }
size_t derivative_workspace(sp_plan_t p, int spectra) {
  // + 256 bytes for the chop's maximum
  return spectra * spectrum_bytes(p) + ((sp::msin_scratch_bytes(p->N, p->Kp) + 255) & ~(size_t)255) + 256;
}
int check_derivative_call(sp_plan_t plan, int spectra, std::initializer_list<const void*> ptrs, void* workspace,
                          size_t workspace_bytes) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  for (const void* q : ptrs)
    if (!q) return SP_ERR_NULL;
  if (!workspace) return SP_ERR_NULL;
  if (plan->batched || plan->precision != SP_FP64 || plan->poles) return SP_ERR_UNSUPPORTED;
  uintptr_t bits = (uintptr_t)workspace;
  for (const void* q : ptrs) bits |= (uintptr_t)q;
  if (bits & 15) return SP_ERR_MISALIGNED;
  if (workspace_bytes < derivative_workspace(plan, spectra)) return SP_ERR_WORKSPACE;
  return on_plan_device(plan);
}
struct DerivSpace {
  cpx<double>* X;   // coefficients of the current input
  cpx<double>* Q;   // (1/sin theta) d/dlambda of it
  cpx<double>* P;   // chunk sums of the division
  cpx<double>* G[3];
  unsigned long long* mx;  // max |X| of the chop
};
DerivSpace derivative_space(sp_plan_t p, void* workspace, int spectra) {
  char* b = static_cast<char*>(workspace);
  const size_t one = spectrum_bytes(p);
  DerivSpace d;
  d.X = reinterpret_cast<cpx<double>*>(b);
  d.Q = reinterpret_cast<cpx<double>*>(b + one);
  for (int c = 0; c < 3; ++c) d.G[c] = c + 2 < spectra ? reinterpret_cast<cpx<double>*>(b + (2 + c) * one) : nullptr;
  d.P = reinterpret_cast<cpx<double>*>(b + spectra * one);
  d.mx = reinterpret_cast<unsigned long long*>(b + spectra * one +
                                               ((sp::msin_scratch_bytes(p->N, p->Kp) + 255) & ~(size_t)255));
  return d;
}
// X = coeffs2(f), Q = (1/sin theta) d/dlambda f in coefficients
void enqueue_derivative_input(sp_plan_t p, const double* f, const DerivSpace& d, bool need_q, cudaStream_t st) {
  enqueue_coeffs2(p, f, d.X, p->K, st);
  if (p->chop > 0.0) sp::launch_coeff_chop(st, d.X, p->N, p->K, p->Kp, d.mx, p->chop);
  if (need_q) sp::launch_msin_div(st, d.X, d.Q, d.P, p->N, p->K, p->Kp);
}
// one launch of the coefficient maps on the current input: each output takes
// one signed component ("+x", "-z": T0, -T2), added to its contents when acc
struct ComboOut {
  cpx<double>* G;
  const char* term;
  bool acc;
};
void enqueue_combo(sp_plan_t p, const DerivSpace& d, std::initializer_list<ComboOut> outs, cudaStream_t st) {
  sp::TangentialCombo tc = {};
  int o = 0;
  for (const ComboOut& c : outs) {
    const int comp = c.term[1] - 'x';
    tc.G[o] = c.G;
    tc.comp[o] = (signed char)comp;
    tc.neg[o] = c.term[0] == '-';
    if (c.acc) tc.acc |= (unsigned char)(1u << o);
    if (comp < 2) tc.need_xy = 1;
    else tc.need_z = 1;
    ++o;
  }
  sp::launch_tangential(st, d.X, d.Q, tc, p->N, p->K, p->Kp);
}
// values on the grid of the coefficients G (destroys G)
void enqueue_values(sp_plan_t p, cpx<double>* G, double* out, cudaStream_t st) {
  launch_theta_inverse_x<double>(p, false, st, G, p->N, p->K, p->Kp, p->cols_per_cta, p->col_fft, p->tw_col,
                                 p->perm_col, p->post_col, 1.0 / p->N, 2);
  launch_rows_inverse_x<double>(p, false, st, G, out, p->nt, p->nl, p->Kp, p->rows_per_cta, p->row_fft,
                                p->tw_row, p->perm_row, p->post_row, p->row_scale, p->row_scale, nullptr);
}
// the coefficients of the three curl components of (f1, f2, f3) into d.G[0..2]:
// (d/dy f3 - d/dz f2, d/dz f1 - d/dx f3, d/dx f2 - d/dy f1)
void enqueue_curl_coefficients(sp_plan_t p, const double* f1, const double* f2, const double* f3,
                               const DerivSpace& d, cudaStream_t st) {
  enqueue_derivative_input(p, f1, d, true, st);
  enqueue_combo(p, d, {{d.G[1], "+z", false}, {d.G[2], "-y", false}}, st);
  enqueue_derivative_input(p, f2, d, true, st);
  enqueue_combo(p, d, {{d.G[0], "-z", false}, {d.G[2], "+x", true}}, st);
  enqueue_derivative_input(p, f3, d, true, st);
  enqueue_combo(p, d, {{d.G[0], "+y", true}, {d.G[1], "-x", true}}, st);
}
int launch_status(const char* what) {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SP_OK : cuda_fail(e, what);
}
}  // namespace

int sphere_poisson_gradient_workspace_size(sp_plan_t plan, size_t* workspace_bytes) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!workspace_bytes) return SP_ERR_NULL;
  if (plan->batched || plan->precision != SP_FP64 || plan->poles) return SP_ERR_UNSUPPORTED;
  *workspace_bytes = derivative_workspace(plan, 5);
  return SP_OK;
}

int sphere_poisson_curl_workspace_size(sp_plan_t plan, size_t* workspace_bytes) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!workspace_bytes) return SP_ERR_NULL;
  if (plan->batched || plan->precision != SP_FP64 || plan->poles) return SP_ERR_UNSUPPORTED;
  *workspace_bytes = derivative_workspace(plan, 5);
  return SP_OK;
}

int sphere_poisson_set_chop(sp_plan_t plan, double rtol) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!(rtol >= 0.0 && rtol < 1.0)) return SP_ERR_BAD_ARG;  // also rejects NaN
  plan->chop = rtol;
  return SP_OK;
}

int sphere_poisson_tangential_gradient(sp_plan_t plan, const double* f, double* gx, double* gy, double* gz,
                                       void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_derivative_call(plan, 5, {f, gx, gy, gz}, workspace, workspace_bytes);
  if (rc != SP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const DerivSpace d = derivative_space(plan, workspace, 5);
  enqueue_derivative_input(plan, f, d, true, st);
  enqueue_combo(plan, d, {{d.G[0], "+x", false}, {d.G[1], "+y", false}, {d.G[2], "+z", false}}, st);
  double* out[3] = {gx, gy, gz};
  for (int c = 0; c < 3; ++c) enqueue_values(plan, d.G[c], out[c], st);
  return launch_status("tangential gradient launch");
}

int sphere_poisson_divergence(sp_plan_t plan, const double* f1, const double* f2, const double* f3, double* div,
                              void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_derivative_call(plan, 3, {f1, f2, f3, div}, workspace, workspace_bytes);
  if (rc != SP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const DerivSpace d = derivative_space(plan, workspace, 3);
  const double* f[3] = {f1, f2, f3};
  const char* terms[3] = {"+x", "+y", "+z"};
  for (int c = 0; c < 3; ++c) {
    enqueue_derivative_input(plan, f[c], d, c < 2, st);  // d/dz needs no division
    enqueue_combo(plan, d, {{d.G[0], terms[c], c > 0}}, st);
  }
  enqueue_values(plan, d.G[0], div, st);
  return launch_status("divergence launch");
}

int sphere_poisson_curl(sp_plan_t plan, const double* f1, const double* f2, const double* f3, double* c1,
                        double* c2, double* c3, void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_derivative_call(plan, 5, {f1, f2, f3, c1, c2, c3}, workspace, workspace_bytes);
  if (rc != SP_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const DerivSpace d = derivative_space(plan, workspace, 5);
  enqueue_curl_coefficients(plan, f1, f2, f3, d, st);
  double* out[3] = {c1, c2, c3};
  for (int c = 0; c < 3; ++c) enqueue_values(plan, d.G[c], out[c], st);
  return launch_status("curl launch");
}

int sphere_poisson_scalar_curl(sp_plan_t plan, const double* f, double* c1, double* c2, double* c3,
                               void* workspace, size_t workspace_bytes, void* stream) {
  int rc = sphere_poisson_tangential_gradient(plan, f, c1, c2, c3, workspace, workspace_bytes, stream);
  if (rc != SP_OK) return rc;
  sp::launch_cross_normal(static_cast<cudaStream_t>(stream), c1, c2, c3, plan->geo, plan->nt, plan->nl);
  return launch_status("scalar curl launch");
}

int sphere_poisson_vorticity(sp_plan_t plan, const double* f1, const double* f2, const double* f3, double* zeta,
                             void* workspace, size_t workspace_bytes, void* stream) {
  int rc = check_derivative_call(plan, 5, {f1, f2, f3, zeta}, workspace, workspace_bytes);
  if (rc != SP_OK) return rc;
  sp_plan_t p = plan;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const DerivSpace d = derivative_space(p, workspace, 5);
  enqueue_curl_coefficients(p, f1, f2, f3, d, st);
  // the first two curl components land in the (now free) X and Q spectra as
  // real grids (N Kp 16 >= n_theta n_lambda 8 bytes), the third in zeta
  double* t1 = reinterpret_cast<double*>(d.X);
  double* t2 = reinterpret_cast<double*>(d.Q);
  enqueue_values(p, d.G[0], t1, st);
  enqueue_values(p, d.G[1], t2, st);
  enqueue_values(p, d.G[2], zeta, st);
  sp::launch_normal_dot(st, t1, t2, zeta, zeta, p->geo, p->nt, p->nl);
  return launch_status("vorticity launch");
}

namespace {
constexpr int kGeParts = 608;  // partial-maximum blocks of the pivot search (4 per SM)
constexpr int kMaxTerms = 1024;  // low-rank terms (the outer product keeps 2 x terms coefficients in shared memory)
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

int sphere_poisson_lowrank_workspace_size(sp_plan_t plan, int max_terms, size_t* workspace_bytes) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!workspace_bytes) return SP_ERR_NULL;
  if (plan->batched || plan->precision != SP_FP64 || plan->poles) return SP_ERR_UNSUPPORTED;
  if (max_terms < 0 || max_terms > std::min(plan->nt, kMaxTerms)) return SP_ERR_BAD_ARG;
  const size_t ge = al256((size_t)plan->nt * plan->nl * sizeof(double)) + al256(kGeParts * sizeof(sp::GePivot)) +
                    al256(sizeof(sp::GePivot)) + al256(2 * (size_t)plan->nl * sizeof(double));
  const size_t sv = al256((size_t)plan->N * plan->Kp * sizeof(cpx<double>)) +
                    al256((size_t)plan->N * 2 * std::max(max_terms, 1) * sizeof(cpx<double>)) +
                    al256((size_t)std::max(max_terms, 1) * plan->Kp * sizeof(cpx<double>));
  *workspace_bytes = std::max(ge, sv);
  return SP_OK;
}

int sphere_poisson_lowrank_ge(sp_plan_t plan, const double* f, int max_terms, double rtol, double alpha,
                              int* terms, double* cols, double* piv, double* rows, void* workspace,
                              size_t workspace_bytes, void* stream) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!f || !terms || !workspace || (max_terms > 0 && (!cols || !piv || !rows))) return SP_ERR_NULL;
  if (plan->batched || plan->precision != SP_FP64 || plan->poles) return SP_ERR_UNSUPPORTED;
  if (max_terms < 0 || max_terms > std::min(plan->nt, kMaxTerms) || !(rtol >= 0.0) || !(alpha >= 0.0) || alpha > 1.0)
    return SP_ERR_BAD_ARG;
  if (((uintptr_t)f | (uintptr_t)workspace) & 15) return SP_ERR_MISALIGNED;
  size_t need = 0;
  sphere_poisson_lowrank_workspace_size(plan, max_terms, &need);
  if (workspace_bytes < need) return SP_ERR_WORKSPACE;
  if (int drc = on_plan_device(plan)) return drc;
  const int nt = plan->nt, n = plan->nl, H = n / 2, m = 2 * nt;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(workspace);
  double* e = reinterpret_cast<double*>(base);
  sp::GePivot* part = reinterpret_cast<sp::GePivot*>(base + al256((size_t)nt * n * sizeof(double)));
  sp::GePivot* pv = reinterpret_cast<sp::GePivot*>(reinterpret_cast<char*>(part) + al256(kGeParts * sizeof(sp::GePivot)));
  double* AB = reinterpret_cast<double*>(reinterpret_cast<char*>(pv) + al256(sizeof(sp::GePivot)));
  *terms = 0;
  cudaError_t err = cudaMemcpyAsync(e, f, (size_t)nt * n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  if (err != cudaSuccess) return cuda_fail(err, "lowrank_ge copy");
  std::vector<double> hpiv;
  double scale = 0.0, best = 1e300;
  int stall = 0, count = 0;
  for (int t = 0; t < max_terms; ++t) {
    sp::launch_ge_pivot(st, e, nt, n, part, kGeParts, pv);
    sp::GePivot hp;
    err = cudaMemcpyAsync(&hp, pv, sizeof hp, cudaMemcpyDeviceToHost, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err != cudaSuccess) return cuda_fail(err, "lowrank_ge pivot");
    if (t == 0) scale = hp.maxabs;
    const double r = hp.maxabs;
    if (r <= rtol * scale) break;
    if (r < best) {
      best = r;
      stall = 0;
    } else if (r < 1e-9 * scale && ++stall >= 3) {
      break;  // the residual has reached its rounding floor
    }
    const int istar = (int)(hp.index / H), qstar = H + (int)(hp.index % H);
    // epsilon-pseudoinverse of [[a, b], [b, a]]: eigenvalues a + b ((1,1)/sqrt2), a - b ((1,-1)/sqrt2)
    const double l1 = hp.a + hp.b, l2 = hp.a - hp.b;
    const double eps = alpha * std::max(std::fabs(l1), std::fabs(l2));
    const double h1 = std::fabs(l1) > eps ? 0.5 / l1 : 0.0, h2 = std::fabs(l2) > eps ? 0.5 / l2 : 0.0;
    const double p0 = h1 + h2, p1 = h1 - h2;
    double* col = cols + (size_t)t * m;
    double* row = rows + (size_t)t * n;
    sp::launch_ge_step(st, e, nt, n, istar, qstar, col, row, p0, p1, AB);
    hpiv.push_back(p0);
    hpiv.push_back(p1);
    ++count;
  }
  if (count) err = cudaMemcpyAsync(piv, hpiv.data(), hpiv.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (err == cudaSuccess) err = cudaStreamSynchronize(st);
  if (err == cudaSuccess) err = cudaGetLastError();
  if (err != cudaSuccess) return cuda_fail(err, "lowrank_ge");
  *terms = count;
  return SP_OK;
}

int sphere_poisson_solve_lowrank(sp_plan_t plan, int terms, const double* cols, const double* piv,
                                 const double* rows, double* u, void* workspace, size_t workspace_bytes,
                                 void* stream) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!u || !workspace || (terms > 0 && (!cols || !piv || !rows))) return SP_ERR_NULL;
  if (plan->batched || plan->precision != SP_FP64 || plan->poles) return SP_ERR_UNSUPPORTED;
  if (terms < 0 || terms > std::min(plan->nt, kMaxTerms)) return SP_ERR_BAD_ARG;
  if (((uintptr_t)u | (uintptr_t)workspace | (uintptr_t)cols | (uintptr_t)rows) & 15) return SP_ERR_MISALIGNED;
  size_t need = 0;
  sphere_poisson_lowrank_workspace_size(plan, terms, &need);
  if (workspace_bytes < need) return SP_ERR_WORKSPACE;
  if (int drc = on_plan_device(plan)) return drc;
  sp_plan_t p = plan;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(workspace);
  cpx<double>* W = reinterpret_cast<cpx<double>*>(base);
  cpx<double>* Wc = reinterpret_cast<cpx<double>*>(base + al256((size_t)p->N * p->Kp * sizeof(cpx<double>)));
  cpx<double>* R = reinterpret_cast<cpx<double>*>(reinterpret_cast<char*>(Wc) +
                                                  al256((size_t)p->N * 2 * std::max(terms, 1) * sizeof(cpx<double>)));
  const double inv_n = 1.0 / (double)p->N;
  if (terms > 0) {
    sp::launch_lowrank_pack(st, cols, terms, p->nt, p->sin2, Wc);
    launch_theta_forward_x<double>(p, false, st, Wc, p->N, 2 * terms, 2 * terms, p->cols_per_cta, p->col_fft,
                                   p->tw_col, p->perm_col, p->post_col_s, inv_n, 1);
    launch_rows_forward_x<double>(p, false, st, rows, R, terms, p->nl, p->Kp, p->rows_per_cta, p->row_fft,
                                  p->tw_row, p->perm_row, p->post_row, p->row_plain, p->row_plain, nullptr);
  }
  sp::launch_lowrank_outer(st, Wc, R, piv, terms, p->N, p->K, p->Kp, W);
  const sp::Launch solve{dim3((p->K + 31) / 32, 2), 32, 0, st};
  sp::launch_solve<double>(false, solve, W, p->fac_l, p->fac_iu, p->fac_cu, p->N, p->K, p->Kp);
  launch_theta_inverse_x<double>(p, false, st, W, p->N, p->K, p->Kp, p->cols_per_cta, p->col_fft, p->tw_col,
                                 p->perm_col, p->post_col, inv_n, 1);
  launch_rows_inverse_x<double>(p, false, st, W, u, p->nt, p->nl, p->Kp, p->rows_per_cta, p->row_fft,
                                p->tw_row, p->perm_row, p->post_row, p->row_scale, p->row_scale, nullptr);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SP_OK : cuda_fail(e, "solve_lowrank launch");
}

int sphere_poisson_launch_count(sp_plan_t plan, int adjoint, int* launches) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!launches) return SP_ERR_NULL;
  if (plan->batched) *launches = (plan->bsplit > 0 ? 1 : 0) + (plan->count > plan->bsplit ? 1 : 0);
  else if (plan->precision == SP_FP64) *launches = kStages;
  else if (plan->precision == SP_FP32)
    *launches = (plan->fused && (!adjoint || plan->fuse_cols < 0) ? kStages - 2 : kStages) + 3;
  else if (adjoint) *launches = 0;
  else *launches = plan->fused ? 3 + 5 : kStages - 1 + 3 + (plan->sweeps + 1);
  return SP_OK;
}

static void release_events(sp_plan_t plan) {
  for (cudaEvent_t e : plan->prof_events) cudaEventDestroy(e);
  plan->prof_events.clear();
  plan->prof_max = plan->prof_count = 0;
}

int sphere_poisson_profile_begin(sp_plan_t plan, int max_solves) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (max_solves < 1 || max_solves > 100000) return SP_ERR_BAD_ARG;
  release_events(plan);
  plan->prof_events.resize((size_t)max_solves * (kStages + 1));
  for (auto& e : plan->prof_events) {
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) {
      e = nullptr;
      release_events(plan);
      return cuda_fail(err, "cudaEventCreate");
    }
  }
  plan->prof_max = max_solves;
  plan->prof_count = 0;
  return SP_OK;
}

int sphere_poisson_profile_end(sp_plan_t plan, double* stage_ms, int max_stages, int* solves, int* stages) {
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  if (!stage_ms || !solves || !stages) return SP_ERR_NULL;
  for (int s = 0; s < max_stages; ++s) stage_ms[s] = 0.0;
  int rc = SP_OK;
  for (int c = 0; c < plan->prof_count && rc == SP_OK; ++c) {
    cudaEvent_t* ev = &plan->prof_events[(size_t)c * (kStages + 1)];
    cudaError_t err = cudaEventSynchronize(ev[kStages]);
    if (err != cudaSuccess) { rc = cuda_fail(err, "cudaEventSynchronize"); break; }
    for (int s = 0; s < kStages && s < max_stages; ++s) {
      float ms = 0.f;
      err = cudaEventElapsedTime(&ms, ev[s], ev[s + 1]);
      if (err != cudaSuccess) { rc = cuda_fail(err, "cudaEventElapsedTime"); break; }
      stage_ms[s] += ms;
    }
  }
  *solves = plan->prof_count;
  *stages = kStages;
  release_events(plan);
  return rc;
}

const char* sphere_poisson_stage_name(sp_plan_t plan, int stage) {
  if (!plan_ok(plan) || stage < 0 || stage >= kStages) return "";
  return plan->fused ? kFusedStageNames[stage] : kStageNames[stage];
}

int sphere_poisson_destroy(sp_plan_t plan) {
  if (!plan) return SP_OK;
  if (!plan_ok(plan)) return SP_ERR_BAD_PLAN;
  release_events(plan);
  destroy_plan(plan);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "sphere_poisson_destroy");
  return SP_OK;
}

const char* sphere_poisson_status_string(int status) {
  switch (status) {
    case SP_OK: return "success";
    case SP_WARN_NONZERO_MEAN: return "warning: f does not have zero mean over the sphere (the paper's assumption); "
                                      "the solve dropped the k = 0, j = 0 equation";
    case SP_ERR_BAD_SIZE: return "bad grid size: need n_theta >= 1, even n_lambda >= 2, lengths <= 12288 "
                                 "with prime factors <= 31";
    case SP_ERR_NULL: return "a required pointer is NULL";
    case SP_ERR_MISALIGNED: return "a device pointer is not 16-byte aligned";
    case SP_ERR_WORKSPACE: return "workspace smaller than the plan requires";
    case SP_ERR_CUDA: return g_cuda_msg[0] ? g_cuda_msg : "CUDA runtime error";
    case SP_ERR_UNSUPPORTED: return "precision or flag combination not supported";
    case SP_ERR_BAD_PLAN: return "NULL or destroyed plan handle";
    case SP_ERR_BAD_ARG: return "invalid argument";
    case SP_ERR_SCRATCH_LIMIT: return "grid too large for the 32 MiB fixed scratch of sphere_poisson_solve_noalloc; "
                                      "use sphere_poisson_solve with a workspace";
    case SP_ERR_TIMEOUT: return "a kernel's bounded wait for its asynchronous copies gave up; the results of the "
                                "solves since the last status check are not valid";
    default: return "unknown status";
  }
}

}  // extern "C"
