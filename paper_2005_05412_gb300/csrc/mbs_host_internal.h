// mbs_host_internal.h -- private declarations shared by the host units of
// the library:
//   mbs_setup.cpp       FP64 linear algebra and the step operators of a quantum
//                       description (Sec. 2.2 splitting, Sec. 3.1.1 relaxation)
//   mbs_host.cpp        objects (device, scenario), their C-ABI calls and
//                       device buffers
//   mbs_solve.cpp       the solve of one scenario, periodic state checks, the
//                       tile-depth autotuner and mbs_solve
//   mbs_batch.cpp       batched solves of many scenarios and their CUDA graphs
//   mbs_cells_host.cpp  driven single cells (Nx = 1)
#pragma once
#include <cuda_runtime.h>

#include <cfloat>
#include <complex>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mbs.h"
#include "mbs_internal.h"

using cd = std::complex<double>;

namespace mbs_host {

constexpr double kPlanck = 6.62607015e-34;  // CODATA 2018
constexpr double kPi = 3.14159265358979323846;
constexpr double kHbar = kPlanck / (2.0 * kPi);
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.25663706212e-6;

// the calling thread's last error message (mbs_last_error)
extern thread_local std::string g_err;
// byte counter of the current host -> device upload phase (or null)
extern thread_local long long *g_h2d;
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// ---------------------------------------------------- FP64 setup (mbs_setup.cpp)
void cmatmul(int n, const cd *a, const cd *b, cd *c);
void rmatmul(int n, const double *a, const double *b, double *c);
std::vector<cd> conj_transform(int n, const std::vector<cd> &X, const cd *A);
bool eigh_hq(int n, const cd *A, double *w, cd *V);
void expm1_taylor(int n, const double *A, double *E);
double solve(int n, std::vector<double> A, std::vector<double> &b);
void herm_to_y(int N, const cd *X, double *y);
void y_to_herm(int N, const double *y, cd *X);
// full index of Bloch-deviation index i (drops rho~_{N-1,N-1})
inline int full_of(int N, int i) { return i < N - 1 ? i : i + 1; }

struct QDesc {
  int N = 0;
  double n3d = 0;
  std::vector<double> lambda;   // eigenvalues of mu
  std::vector<cd> V;            // eigenvectors (columns)
  std::vector<double> MH, MD;   // generator parts on full coords (N^2 x N^2)
  std::vector<double> yref, yinit;
  bool unique_steady = false;
};

struct Step {  // FP64 step operators for one (description, H0 factor)
  std::vector<double> AK;    // exp(L0 dt) on Bloch deviations
  std::vector<double> AKm1;  // the same minus I, formed without cancellation
  std::vector<double> c, g, Ah;
  std::vector<double> Ehm1;  // exp(L0 dt/2) - I on the full coordinates
  double g0 = 0;
};

void build_step(const QDesc &q, double hfac, double dt, Step &s);
std::vector<double> rho_functional(const QDesc &q, int a, int b, bool im);
bool herm_ok(int n, const double *m, double tol_rel);
std::vector<cd> load(int n, const double *m);
int build_qdesc(const mbs_qm_desc &in, QDesc &q);

struct MatDesc {
  double eps_r, mu_r, sigma, overlap;
  int qm;
};
struct SrcHost {
  int kind, face, cell;
  std::vector<double> sH, sE;
};

struct Bundle {  // device buffers of one precision
  bool ready = false;
  size_t rb = 8;
  void *E[2] = {}, *H[2] = {}, *El[2] = {}, *Hl[2] = {}, *D[2] = {}, *C[2] = {}, *pd = nullptr, *Dinit = nullptr;
  void *emc = nullptr, *qpar = nullptr, *pcell = nullptr, *pcell2 = nullptr, *pr_coef = nullptr, *rec = nullptr;
  float *tcw = nullptr;
  void *bprev[2] = {};   // E_b^{n-1} of the two ends at a launch boundary: [left hi, left lo, right hi, right lo]
  std::vector<void *> src_tabs;
};

}  // namespace mbs_host

// ------------------------------------------------------------ objects
struct mbs_device_s {
  std::vector<mbs_host::QDesc> qms;
  std::vector<mbs_host::MatDesc> mats;
  int nx = 0;
  double length = 0, dz = 0;
  int bc_l = 0, bc_r = 0;   // 0 Mur, 1 mirror, 2 partial
  double r_l = 0, r_r = 0;  // amplitude reflections -sqrt(R)
  std::vector<uint8_t> cell_mat;   // [nx]
  std::vector<double> jitter;      // [nx][2] or empty
  int N = 0;                       // common level count of the media (0: none)
};

struct mbs_scenario_s {
  mbs_device_s *dev = nullptr;
  double dt = 0;
  long long nt = 0;
  int N = 0, K = 0, P = 0;
  int ld = 0, off = mbs::PAD;
  int n_slot = 0, qstride = 0;
  // FP64 master copies
  std::vector<double> emc, qpar, pcell, pcell2, Dinit, pr_coef, zref;
  std::vector<float> tcw;  // tensor-core tiles' constant table (N >= 4, one medium)
  std::vector<double> e_init;  // initial field E^0 [nx] (empty: zero)
  // host staging of the asynchronous reset copies (kept alive until the next reset)
  std::vector<float> e_init_f, bprev_init_f = std::vector<float>(4);
  std::vector<double> bprev_init_d = std::vector<double>(4);
  bool has_b2 = false;   // structured two-level rows available (pcell2)

  std::vector<int> qslot, pr_cell, pr_q;
  std::vector<mbs_host::SrcHost> src;
  double kmur_l = 0, kmur_r = 0;
  bool has_pcell = false;
  // jittered two-level media set up on the device: the FP64 per-cell rows
  // ([pc_rows][ld], [7][ld], [3][ld]); the bundles copy or convert them
  double *d_pcell64 = nullptr, *d_pcell2_64 = nullptr, *d_dinit64 = nullptr;
  // device
  uint8_t *d_mat = nullptr;
  int *d_qslot = nullptr, *d_pr_cell = nullptr, *d_pr_q = nullptr, *d_flags = nullptr, *d_chk_cells = nullptr;
  double *d_zref = nullptr, *d_chk_min = nullptr, *d_chk_tr = nullptr;
  std::vector<int> chk_cells;
  mbs_host::Bundle b[2];
  int solved_prec = -1, last_cur = 0;
  int tile_used = 0;   // tile depth of the last solve (0: plain path)
  int tc_cells = 128;  // cells per tensor-core tile of the current solve (N >= 4)
  long long h2d_bytes = 0, d2h_bytes = 0, launches = 0;
  long long steps_run = 0;
  double st_trace = 0, st_min = 0;
  int device_id = 0;
};

namespace mbs_host {

// ------------------------------------------------- device buffers (mbs_host.cpp)
size_t rsize(int prec);
int upload(const std::vector<double> &h, void **dptr, int prec);
int upload_src(const std::vector<double> &h, void **dptr, int prec);
template <typename T>
int upload_raw(const std::vector<T> &h, T **dptr) {
  if (h.empty()) {
    *dptr = nullptr;
    return 0;
  }
  if (g_h2d) *g_h2d += (long long)(h.size() * sizeof(T));
  cudaError_t e = cudaMalloc((void **)dptr, h.size() * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  e = cudaMemcpy(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  return 0;
}
void free_bundle(Bundle &b);
int ensure_bundle(mbs_scenario_s *s, int prec);
mbs::Args make_args(mbs_scenario_s *s, int prec);
void free_scenario(mbs_scenario_s *s);
double light_speed(const MatDesc &m);
double envelope(int shape, double x);

// ---------------------------------------------------- solving (mbs_solve.cpp)
int prepare_solve(mbs_scenario_s *s, int prec, cudaStream_t st);
int default_tile_steps(int N, int tc_cells = 128);
bool uses_tc(const mbs_scenario_s *s, int prec);
int default_algo(const mbs_scenario_s *s, int prec);
int tiled_ok(const mbs_scenario_s *s, int prec, int T);
int launch_state_check(mbs_scenario_s *s, const mbs::Args &a, int c, cudaStream_t st);
int periodic_check(mbs_scenario_s *s, const mbs::Args &a, int dcur, int ecur, int hcur, cudaStream_t st, bool wait,
                   bool *failed);
int finish_solve(mbs_scenario_s *s, int prec, int cur, long long steps_run = -1);
int solve_one(mbs_scenario_s *s, const mbs_opts &o, cudaStream_t st);
// tile-depth autotuner: candidates, and the cache of measured choices
std::vector<int> tile_candidates(int N, long long nt);
extern std::mutex g_tune_mu;
extern std::map<std::string, int> g_tune;
// code of a measured candidate: the tile depth, plus 1000 for 256-cell
// tensor-core tiles
inline int code_steps(int code) { return code % 1000; }
inline int code_cells(int code) { return code >= 1000 ? 256 : 128; }
// time `run(code, cur)` (which enqueues one launch) for every candidate; -1
// on error
template <class Run>
int tune_loop(const std::vector<int> &cands, cudaStream_t st, Run run) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return -1;
  }
  int best = -1;
  float best_t = FLT_MAX;
  for (int T : cands) {
    bool ok = run(T, 0) == 0;
    float ms = FLT_MAX;   // the faster of two rounds of three launches
    for (int round = 0; round < 2 && ok; ++round) {
      ok = cudaEventRecord(e0, st) == cudaSuccess;
      for (int r = 0; r < 3 && ok; ++r) ok = run(T, (r + 1) & 1) == 0;
      ok = ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
      float m = 0;
      ok = ok && cudaEventElapsedTime(&m, e0, e1) == cudaSuccess;
      ms = std::min(ms, m);
    }
    if (!ok) {
      best = -1;
      break;
    }
    const float per_step = ms / (3.0f * code_steps(T));
    if (per_step < best_t) {
      best_t = per_step;
      best = T;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}


// ------------------------------------------------ batched solves (mbs_batch.cpp)
int solve_batch(std::vector<mbs_scenario_s *> &ss, const mbs_opts &o, cudaStream_t st);
void drop_graphs_of(mbs_scenario_s *s);   // frees the batched-solve graphs that use s

}  // namespace mbs_host
