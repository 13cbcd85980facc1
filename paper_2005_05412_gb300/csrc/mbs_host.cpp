// mbs_host.cpp -- host side of the GB300 Maxwell-Bloch hot path: C-ABI
// entry points (include/mbs.h), input validation, the FP64 setup of the
// per-material step operators, device buffers and the solve loop.
//
// FP64 setup per quantum description (Sec. 2.2 operator splitting, Sec. 3.1
// Lindblad relaxation):
//   * mu = V diag(lambda) V^+ by Householder reduction of the Hermitian
//     matrix to real symmetric tridiagonal form followed by implicit QL
//     iterations (Golub & Van Loan, Secs. 8.3 and 8.5);
//   * the Liouvillian L0 (H0 and the dissipator of Eq. lindbladdiss) as a
//     real matrix on the coordinates of rho~ = V^+ rho V (mbs_internal.h);
//     the rate form (Eq. relax_pop, pure dephasing) becomes Lindblad
//     operators |i><j| and diag(v_k), the latter from the double-centred
//     dephasing matrix G = -1/2 J D J (D_ij = 2 gamma_ij,p), which is PSD iff
//     the dephasing rates admit a PSD coefficient matrix;
//   * exp(L0 dt) and exp(L0 dt/2) by Taylor series with scaling and
//     squaring;
//   * the steady state of L0 (when unique) as the deviation reference.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cfloat>
#include <climits>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "../../include/mbs.h"
#include "mbs_internal.h"

using cd = std::complex<double>;

namespace {

constexpr double kPlanck = 6.62607015e-34;  // CODATA 2018
constexpr double kPi = 3.14159265358979323846;
constexpr double kHbar = kPlanck / (2.0 * kPi);
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.25663706212e-6;

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? MBS_E_OOM : MBS_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------ linear algebra
void cmatmul(int n, const cd *a, const cd *b, cd *c) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      cd s = 0;
      for (int k = 0; k < n; ++k) s += a[i * n + k] * b[k * n + j];
      c[i * n + j] = s;
    }
}

void rmatmul(int n, const double *a, const double *b, double *c) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0;
      for (int k = 0; k < n; ++k) s += a[i * n + k] * b[k * n + j];
      c[i * n + j] = s;
    }
}

// X^+ A X for n x n complex matrices
std::vector<cd> conj_transform(int n, const std::vector<cd> &X, const cd *A) {
  std::vector<cd> t(n * n), xh(n * n), out(n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) xh[i * n + j] = std::conj(X[j * n + i]);
  cmatmul(n, xh.data(), A, t.data());
  cmatmul(n, t.data(), X.data(), out.data());
  return out;
}

// Hermitian eigen-decomposition (ascending eigenvalues, eigenvectors in the
// columns of V): Householder reduction to Hermitian tridiagonal form, a
// diagonal phase change to real symmetric tridiagonal, implicit QL with
// Wilkinson-type shifts on (d, e).
bool eigh_hq(int n, const cd *A, double *w, cd *V) {
  std::vector<cd> a(A, A + n * n), Q(n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
  std::vector<cd> v(n);
  for (int k = 0; k + 2 < n; ++k) {
    double xn = 0;
    for (int i = k + 1; i < n; ++i) xn += std::norm(a[i * n + k]);
    xn = std::sqrt(xn);
    if (xn == 0) continue;
    const cd x0 = a[(k + 1) * n + k];
    const cd ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1.0);
    const cd alpha = -ph * xn;
    std::fill(v.begin(), v.end(), cd(0));
    for (int i = k + 1; i < n; ++i) v[i] = a[i * n + k];
    v[k + 1] -= alpha;
    double vn = 0;
    for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
    if (vn == 0) continue;
    const double f = 2.0 / vn;
    for (int j = 0; j < n; ++j) {  // a <- (I - f v v^+) a
      cd s = 0;
      for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * a[i * n + j];
      for (int i = k + 1; i < n; ++i) a[i * n + j] -= f * v[i] * s;
    }
    for (int i = 0; i < n; ++i) {  // a <- a (I - f v v^+), Q <- Q (I - f v v^+)
      cd s = 0, sq = 0;
      for (int j = k + 1; j < n; ++j) {
        s += a[i * n + j] * v[j];
        sq += Q[i * n + j] * v[j];
      }
      for (int j = k + 1; j < n; ++j) {
        a[i * n + j] -= f * s * std::conj(v[j]);
        Q[i * n + j] -= f * sq * std::conj(v[j]);
      }
    }
  }
  // phases making the sub-diagonal real and non-negative
  std::vector<double> d(n), e(n, 0.0);
  std::vector<cd> ph(n, 1.0);
  for (int k = 0; k < n; ++k) d[k] = a[k * n + k].real();
  for (int k = 0; k + 1 < n; ++k) {
    const cd b = a[(k + 1) * n + k];
    const double r = std::abs(b);
    e[k] = r;
    ph[k + 1] = r > 0 ? ph[k] * (b / r) : ph[k];
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) Q[i * n + k] *= ph[k];
  // implicit QL on the symmetric tridiagonal (d, e); Z accumulates rotations
  std::vector<double> z(n * n, 0.0);
  for (int i = 0; i < n; ++i) z[i * n + i] = 1.0;
  for (int l = 0; l < n; ++l) {
    int iter = 0;
    for (;;) {
      int m = l;
      for (; m + 1 < n; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= DBL_EPSILON * dd) break;
      }
      if (m == l) break;
      if (++iter > 100) return false;
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + std::copysign(r, g));
      double s = 1.0, c = 1.0, p = 0.0;
      int i = m - 1;
      bool early = false;
      for (; i >= l; --i) {
        double f = s * e[i];
        const double b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[m] = 0.0;
          early = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        for (int k = 0; k < n; ++k) {
          f = z[k * n + i + 1];
          z[k * n + i + 1] = s * z[k * n + i] + c * f;
          z[k * n + i] = c * z[k * n + i] - s * f;
        }
      }
      if (early) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int x, int y) { return d[x] < d[y]; });
  for (int k = 0; k < n; ++k) {
    w[k] = d[ord[k]];
    for (int i = 0; i < n; ++i) {
      cd s = 0;
      for (int j = 0; j < n; ++j) s += Q[i * n + j] * z[j * n + ord[k]];
      V[i * n + k] = s;
    }
  }
  return true;
}

// exp(A) - I for a real n x n matrix, accurate relative to itself: scale by
// 2^-s until ||A||_1 <= 1/4, sum the Taylor series without its leading
// identity to order 20 (remainder < 1e-32 relative), and undo the scaling
// with the squarings in the same form, exp(2B) - I = E (E + 2 I) for
// E = exp(B) - I.  The step operators act on small deviations through
// exp(L0 dt) - I, whose entries are ~|L0| dt; forming exp(L0 dt) first and
// subtracting I would leave them with an absolute error of one ulp of 1 --
// a systematic error repeated every step.
void expm1_taylor(int n, const double *A, double *E) {
  double nrm = 0;
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += std::fabs(A[i * n + j]);
    nrm = std::max(nrm, s);
  }
  if (!std::isfinite(nrm)) {
    for (int i = 0; i < n * n; ++i) E[i] = std::nan("");
    return;
  }
  int sq = 0;
  while (nrm > 0.25) {
    nrm *= 0.5;
    ++sq;
  }
  const double sc = std::ldexp(1.0, -sq);
  std::vector<double> B(n * n), term(n * n), t2(n * n);
  for (int i = 0; i < n * n; ++i) B[i] = term[i] = E[i] = A[i] * sc;
  for (int k = 2; k <= 20; ++k) {
    rmatmul(n, term.data(), B.data(), t2.data());
    for (int i = 0; i < n * n; ++i) {
      term[i] = t2[i] / k;
      E[i] += term[i];
    }
  }
  for (int k = 0; k < sq; ++k) {
    rmatmul(n, E, E, t2.data());
    for (int i = 0; i < n * n; ++i) E[i] = t2[i] + 2.0 * E[i];
  }
}

// Solve A x = b (n x n, partial pivoting).  Returns the smallest |pivot|
// relative to max |A|, or -1 on exact singularity.
double solve(int n, std::vector<double> A, std::vector<double> &b) {
  double amax = 0;
  for (double x : A) amax = std::max(amax, std::fabs(x));
  double pmin = 1e300;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > std::fabs(A[p * n + k])) p = i;
    if (A[p * n + k] == 0) return -1;
    pmin = std::min(pmin, std::fabs(A[p * n + k]));
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
      std::swap(b[k], b[p]);
    }
    for (int i = k + 1; i < n; ++i) {
      const double f = A[i * n + k] / A[k * n + k];
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; --k) {
    double s = b[k];
    for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * b[j];
    b[k] = s / A[k * n + k];
  }
  return amax > 0 ? pmin / amax : 0;
}

// ------------------------------------------------- real coordinates of rho~
// y[k] = rho~_kk (k < N); pair q = (j, k), j < k: y[N+2q] = Re, y[N+2q+1] = Im
void herm_to_y(int N, const cd *X, double *y) {
  for (int k = 0; k < N; ++k) y[k] = X[k * N + k].real();
  int q = 0;
  for (int j = 0; j < N; ++j)
    for (int k = j + 1; k < N; ++k, ++q) {
      y[N + 2 * q] = X[j * N + k].real();
      y[N + 2 * q + 1] = X[j * N + k].imag();
    }
}

void y_to_herm(int N, const double *y, cd *X) {
  for (int i = 0; i < N * N; ++i) X[i] = 0;
  for (int k = 0; k < N; ++k) X[k * N + k] = y[k];
  int q = 0;
  for (int j = 0; j < N; ++j)
    for (int k = j + 1; k < N; ++k, ++q) {
      X[j * N + k] = cd(y[N + 2 * q], y[N + 2 * q + 1]);
      X[k * N + j] = cd(y[N + 2 * q], -y[N + 2 * q + 1]);
    }
}

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

void build_step(const QDesc &q, double hfac, double dt, Step &s) {
  const int N = q.N, N2 = N * N, K = N2 - 1;
  std::vector<double> M(N2 * N2), Mh(N2 * N2), Eh(N2 * N2), Em1(N2 * N2);
  for (int i = 0; i < N2 * N2; ++i) M[i] = hfac * q.MH[i] + q.MD[i];
  for (int i = 0; i < N2 * N2; ++i) Mh[i] = 0.5 * dt * M[i];
  // exp(L0 dt/2) - I, and exp(L0 dt) - I = Eh (Eh + 2 I)
  expm1_taylor(N2, Mh.data(), Eh.data());
  rmatmul(N2, Eh.data(), Eh.data(), Em1.data());
  for (int i = 0; i < N2 * N2; ++i) Em1[i] += 2.0 * Eh[i];
  s.Ah = Eh;
  for (int i = 0; i < N2; ++i) s.Ah[i * N2 + i] += 1.0;
  s.Ehm1 = Eh;
  // deviation coordinates drop rho~_{N-1,N-1} = 1 - sum of the others:
  // (A - I)_ij = Em1[fi][fj] - Em1[fi][N-1] for population columns j
  s.AKm1.assign(K * K, 0.0);
  s.AK.assign(K * K, 0.0);
  for (int i = 0; i < K; ++i)
    for (int j = 0; j < K; ++j) {
      const int fi = full_of(N, i), fj = full_of(N, j);
      s.AKm1[i * K + j] = Em1[fi * N2 + fj] - (j < N - 1 ? Em1[fi * N2 + N - 1] : 0.0);
      s.AK[i * K + j] = s.AKm1[i * K + j] + (i == j ? 1.0 : 0.0);
    }
  // affine offset at the reference state: (A - I) yref
  std::vector<double> ay(N2, 0.0);
  for (int i = 0; i < N2; ++i)
    for (int j = 0; j < N2; ++j) ay[i] += Em1[i * N2 + j] * q.yref[j];
  s.c.assign(K, 0.0);
  for (int i = 0; i < K; ++i) s.c[i] = ay[full_of(N, i)];
  // d_t P / n3D = tr(mu L0 exp(L0 dt/2) v) = sum_j lambda_j [M Ah y]_j
  std::vector<double> MAh(N2 * N2);
  rmatmul(N2, M.data(), s.Ah.data(), MAh.data());
  std::vector<double> gf(N2, 0.0);
  for (int j = 0; j < N; ++j)
    for (int c = 0; c < N2; ++c) gf[c] += q.lambda[j] * MAh[j * N2 + c];
  s.g.assign(K, 0.0);
  for (int i = 0; i < K; ++i) s.g[i] = gf[full_of(N, i)] - (i < N - 1 ? gf[N - 1] : 0.0);
  s.g0 = 0;
  for (int c = 0; c < N2; ++c) s.g0 += gf[c] * q.yref[c];
}

// Lab-basis functional rho_ab = h . y (real part if im == 0, imaginary part
// otherwise) on the full coordinates.
std::vector<double> rho_functional(const QDesc &q, int a, int b, bool im) {
  const int N = q.N;
  std::vector<double> h(N * N, 0.0);
  auto put = [&](int idx, cd v) { h[idx] = im ? v.imag() : v.real(); };
  for (int j = 0; j < N; ++j) put(j, q.V[a * N + j] * std::conj(q.V[b * N + j]));
  int p = 0;
  for (int j = 0; j < N; ++j)
    for (int k = j + 1; k < N; ++k, ++p) {
      const cd x = q.V[a * N + j] * std::conj(q.V[b * N + k]);
      const cd y = q.V[a * N + k] * std::conj(q.V[b * N + j]);
      put(N + 2 * p, x + y);
      put(N + 2 * p + 1, cd(0, 1) * (x - y));
    }
  return h;
}

}  // namespace

// ============================================================ objects
struct MatDesc {
  double eps_r, mu_r, sigma, overlap;
  int qm;
};

struct mbs_device_s {
  std::vector<QDesc> qms;
  std::vector<MatDesc> mats;
  int nx = 0;
  double length = 0, dz = 0;
  int bc_l = 0, bc_r = 0;   // 0 Mur, 1 mirror, 2 partial
  double r_l = 0, r_r = 0;  // amplitude reflections -sqrt(R)
  std::vector<uint8_t> cell_mat;   // [nx]
  std::vector<double> jitter;      // [nx][2] or empty
  int N = 0;                       // common level count of the media (0: none)
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
  std::vector<SrcHost> src;
  double kmur_l = 0, kmur_r = 0;
  bool has_pcell = false;
  // device
  uint8_t *d_mat = nullptr;
  int *d_qslot = nullptr, *d_pr_cell = nullptr, *d_pr_q = nullptr, *d_flags = nullptr, *d_chk_cells = nullptr;
  double *d_zref = nullptr, *d_chk_min = nullptr, *d_chk_tr = nullptr;
  std::vector<int> chk_cells;
  Bundle b[2];
  int solved_prec = -1, last_cur = 0;
  int tile_used = 0;   // tile depth of the last solve (0: plain path)
  int tc_cells = 128;  // cells per tensor-core tile of the current solve (N >= 4)
  long long h2d_bytes = 0, d2h_bytes = 0, launches = 0;
  long long steps_run = 0;
  double st_trace = 0, st_min = 0;
  int device_id = 0;
};

static void drop_graphs_of(mbs_scenario_s *s);   // batched-solve graphs that use s

namespace {

bool herm_ok(int n, const double *m, double tol_rel) {
  double mx = 0;
  for (int i = 0; i < 2 * n * n; ++i) mx = std::max(mx, std::fabs(m[i]));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double dr = m[2 * (i * n + j)] - m[2 * (j * n + i)];
      const double di = m[2 * (i * n + j) + 1] + m[2 * (j * n + i) + 1];
      if (std::fabs(dr) > tol_rel * mx || std::fabs(di) > tol_rel * mx) return false;
    }
  return true;
}

std::vector<cd> load(int n, const double *m) {
  std::vector<cd> v(n * n);
  for (int i = 0; i < n * n; ++i) v[i] = cd(m[2 * i], m[2 * i + 1]);
  return v;
}

// Build one quantum description; returns MBS_OK / MBS_W_NOT_PSD / error.
int build_qdesc(const mbs_qm_desc &in, QDesc &q) {
  const int N = in.n_levels;
  if (N < 2 || N > mbs::NMAX) return fail(MBS_E_INVALID, "n_levels %d outside [2, %d]", N, mbs::NMAX);
  if (!in.h0 || !in.mu || !in.rho_init) return fail(MBS_E_INVALID, "h0, mu and rho_init are required");
  if (!(in.density >= 0)) return fail(MBS_E_INVALID, "negative density");
  if (!herm_ok(N, in.h0, 1e-12)) return fail(MBS_E_INVALID, "h0 is not Hermitian");
  if (!herm_ok(N, in.mu, 1e-12)) return fail(MBS_E_INVALID, "mu is not Hermitian");
  if (!herm_ok(N, in.rho_init, 1e-12)) return fail(MBS_E_INVALID, "rho_init is not Hermitian");
  if (in.n_lindblad < 0 || (in.n_lindblad > 0 && (!in.lindblad_rates || !in.lindblad_ops)))
    return fail(MBS_E_INVALID, "Lindblad operators missing");
  for (int k = 0; k < in.n_lindblad; ++k)
    if (!(in.lindblad_rates[k] >= 0)) return fail(MBS_E_INVALID, "negative Lindblad rate");
  if (in.scattering)
    for (int i = 0; i < N * N; ++i)
      if (i % (N + 1) != 0 && !(in.scattering[i] >= 0)) return fail(MBS_E_INVALID, "negative scattering rate");
  if (in.pure_dephasing)
    for (int i = 0; i < N * (N - 1) / 2; ++i)
      if (!(in.pure_dephasing[i] >= 0)) return fail(MBS_E_INVALID, "negative pure dephasing rate");
  q.N = N;
  q.n3d = in.density;
  std::vector<cd> h0 = load(N, in.h0), mu = load(N, in.mu), rho0 = load(N, in.rho_init);
  cd tr = 0;
  for (int i = 0; i < N; ++i) tr += rho0[i * N + i];
  if (std::abs(tr - 1.0) > 1e-12) return fail(MBS_E_INVALID, "trace of rho_init is not 1");
  {
    std::vector<double> w(N);
    std::vector<cd> vv(N * N);
    if (!eigh_hq(N, rho0.data(), w.data(), vv.data())) return fail(MBS_E_INVALID, "eig(rho_init) failed");
    if (w[0] < -1e-12) return fail(MBS_E_INVALID, "rho_init is not positive semidefinite");
  }
  q.lambda.assign(N, 0.0);
  q.V.assign(N * N, 0.0);
  if (!eigh_hq(N, mu.data(), q.lambda.data(), q.V.data())) return fail(MBS_E_INVALID, "eig(mu) failed");

  // Lindblad operators in the lab basis
  std::vector<std::vector<cd>> ops;
  std::vector<double> rates;
  for (int k = 0; k < in.n_lindblad; ++k) {
    ops.push_back(load(N, in.lindblad_ops + (size_t)2 * N * N * k));
    rates.push_back(in.lindblad_rates[k]);
  }
  int status = MBS_OK;
  if (in.scattering)
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j)
        if (i != j && in.scattering[i * N + j] > 0) {
          std::vector<cd> op(N * N, 0.0);
          op[i * N + j] = 1.0;
          ops.push_back(op);
          rates.push_back(in.scattering[i * N + j]);
        }
  if (in.pure_dephasing) {
    // G = -1/2 J D J with D_ij = 2 gamma_ij,p: then 1/2 (G_ii + G_jj - 2 G_ij)
    // = gamma_ij,p, and diag ops v_k with rates g_k (G = sum g_k v_k v_k^T)
    // give exactly -gamma_ij,p on rho_ij.
    std::vector<double> D(N * N, 0.0), G(N * N, 0.0);
    int p = 0;
    for (int j = 1; j < N; ++j)
      for (int i = 0; i < j; ++i, ++p) D[i * N + j] = D[j * N + i] = 2.0 * in.pure_dephasing[p];
    std::vector<double> rm(N, 0.0);
    double all = 0;
    for (int i = 0; i < N; ++i) {
      for (int j = 0; j < N; ++j) rm[i] += D[i * N + j] / N;
      all += rm[i] / N;
    }
    double gmax = 0;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        G[i * N + j] = -0.5 * (D[i * N + j] - rm[i] - rm[j] + all);
        gmax = std::max(gmax, std::fabs(G[i * N + j]));
      }
    std::vector<cd> Gc(G.begin(), G.end()), Gv(N * N);
    std::vector<double> gw(N);
    if (!eigh_hq(N, Gc.data(), gw.data(), Gv.data())) return fail(MBS_E_INVALID, "eig(G) failed");
    for (int k = 0; k < N; ++k) {
      if (gw[k] < -1e-12 * gmax) status = MBS_W_NOT_PSD;
      if (std::fabs(gw[k]) <= 1e-14 * gmax) continue;
      std::vector<cd> op(N * N, 0.0);
      for (int i = 0; i < N; ++i) op[i * N + i] = Gv[i * N + k].real();
      ops.push_back(op);
      rates.push_back(gw[k]);
    }
  }

  // generators in the dipole eigenbasis, column by column
  const int N2 = N * N;
  std::vector<cd> Ht = conj_transform(N, q.V, h0.data());
  std::vector<std::vector<cd>> Lt, LL;
  for (auto &op : ops) {
    Lt.push_back(conj_transform(N, q.V, op.data()));
    std::vector<cd> lh(N2), ll(N2);
    const auto &L = Lt.back();
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) lh[i * N + j] = std::conj(L[j * N + i]);
    cmatmul(N, lh.data(), L.data(), ll.data());
    LL.push_back(ll);
  }
  q.MH.assign(N2 * N2, 0.0);
  q.MD.assign(N2 * N2, 0.0);
  std::vector<double> e(N2), col(N2);
  std::vector<cd> X(N2), T1(N2), T2(N2), R(N2), lh(N2);
  for (int c = 0; c < N2; ++c) {
    std::fill(e.begin(), e.end(), 0.0);
    e[c] = 1.0;
    y_to_herm(N, e.data(), X.data());
    cmatmul(N, Ht.data(), X.data(), T1.data());
    cmatmul(N, X.data(), Ht.data(), T2.data());
    for (int i = 0; i < N2; ++i) R[i] = cd(0, -1.0 / kHbar) * (T1[i] - T2[i]);
    herm_to_y(N, R.data(), col.data());
    for (int i = 0; i < N2; ++i) q.MH[i * N2 + c] = col[i];
    std::fill(R.begin(), R.end(), cd(0));
    for (size_t k = 0; k < Lt.size(); ++k) {
      const auto &L = Lt[k];
      for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) lh[i * N + j] = std::conj(L[j * N + i]);
      cmatmul(N, L.data(), X.data(), T1.data());
      cmatmul(N, T1.data(), lh.data(), T2.data());
      for (int i = 0; i < N2; ++i) R[i] += rates[k] * T2[i];
      cmatmul(N, LL[k].data(), X.data(), T1.data());
      cmatmul(N, X.data(), LL[k].data(), T2.data());
      for (int i = 0; i < N2; ++i) R[i] -= 0.5 * rates[k] * (T1[i] + T2[i]);
    }
    herm_to_y(N, R.data(), col.data());
    for (int i = 0; i < N2; ++i) q.MD[i * N2 + c] = col[i];
  }
  // reference state: the steady state of L0 if unique, else rho_init
  q.yinit.assign(N2, 0.0);
  {
    std::vector<cd> rt = conj_transform(N, q.V, rho0.data());
    herm_to_y(N, rt.data(), q.yinit.data());
  }
  std::vector<double> M(N2 * N2), b(N2, 0.0);
  for (int i = 0; i < N2 * N2; ++i) M[i] = q.MH[i] + q.MD[i];
  for (int c = 0; c < N2; ++c) M[(N - 1) * N2 + c] = c < N ? 1.0 : 0.0;  // trace row
  b[N - 1] = 1.0;
  const double piv = solve(N2, M, b);
  q.unique_steady = piv > 1e-9;
  q.yref = q.unique_steady ? b : q.yinit;
  return status;
}

size_t rsize(int prec) { return prec == 0 ? sizeof(double) : sizeof(float); }

thread_local long long *g_h2d = nullptr;   // byte counter of the current upload phase

// upload a double vector as `prec` reals
int upload(const std::vector<double> &h, void **dptr, int prec) {
  const size_t n = h.size();
  if (n == 0) {
    *dptr = nullptr;
    return 0;
  }
  cudaError_t e = cudaMalloc(dptr, n * rsize(prec));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  if (g_h2d) *g_h2d += (long long)(n * rsize(prec));
  if (prec == 0) {
    e = cudaMemcpy(*dptr, h.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  } else {
    std::vector<float> f(n);
    for (size_t i = 0; i < n; ++i) f[i] = (float)h[i];
    e = cudaMemcpy(*dptr, f.data(), n * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  return 0;
}

// per-step source table: FP64 as is; FP32 as [2][nt] high and low words of
// each value (v = hi + lo to ~2^-48 relative)
int upload_src(const std::vector<double> &h, void **dptr, int prec) {
  if (prec == 0) return upload(h, dptr, 0);
  const size_t n = h.size();
  std::vector<float> f(2 * n);
  for (size_t i = 0; i < n; ++i) {
    f[i] = (float)h[i];
    f[n + i] = (float)(h[i] - (double)f[i]);
  }
  cudaError_t e = cudaMalloc(dptr, f.size() * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  if (g_h2d) *g_h2d += (long long)(f.size() * sizeof(float));
  e = cudaMemcpy(*dptr, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  return 0;
}

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

void free_bundle(Bundle &b) {
  for (int i = 0; i < 2; ++i) {
    cudaFree(b.E[i]);
    cudaFree(b.H[i]);
    cudaFree(b.El[i]);
    cudaFree(b.Hl[i]);
    cudaFree(b.D[i]);
    cudaFree(b.C[i]);
  }
  cudaFree(b.pd);
  cudaFree(b.Dinit);
  cudaFree(b.emc);
  cudaFree(b.qpar);
  cudaFree(b.pcell);
  cudaFree(b.pcell2);
  cudaFree(b.pr_coef);
  cudaFree(b.rec);
  cudaFree(b.tcw);
  cudaFree(b.bprev[0]);
  cudaFree(b.bprev[1]);
  for (void *p : b.src_tabs) cudaFree(p);
  b = Bundle();
}

int ensure_bundle(mbs_scenario_s *s, int prec) {
  Bundle &b = s->b[prec];
  if (b.ready) return 0;
  const size_t rb = rsize(prec);
  b.rb = rb;
  const size_t row = (size_t)s->ld * rb;
  const int K = s->K;
  cudaError_t e;
  for (int i = 0; i < 2; ++i) {
    if ((e = cudaMalloc(&b.E[i], row)) != cudaSuccess) return cuda_fail(e, "cudaMalloc E");
    if ((e = cudaMalloc(&b.H[i], row)) != cudaSuccess) return cuda_fail(e, "cudaMalloc H");
    if (prec == 1) {
      if ((e = cudaMalloc(&b.El[i], row)) != cudaSuccess) return cuda_fail(e, "cudaMalloc El");
      if ((e = cudaMalloc(&b.Hl[i], row)) != cudaSuccess) return cuda_fail(e, "cudaMalloc Hl");
    }
    if ((e = cudaMalloc(&b.D[i], row * std::max(K, 1))) != cudaSuccess) return cuda_fail(e, "cudaMalloc D");
    if ((e = cudaMalloc(&b.C[i], row * std::max(K, 1))) != cudaSuccess) return cuda_fail(e, "cudaMalloc C");
  }
  if ((e = cudaMalloc(&b.pd, row)) != cudaSuccess) return cuda_fail(e, "cudaMalloc pd");
  for (int i = 0; i < 2; ++i)
    if ((e = cudaMalloc(&b.bprev[i], 4 * rb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc bprev");
  int rc;
  if ((rc = upload(s->Dinit, &b.Dinit, prec))) return rc;
  if ((rc = upload(s->emc, &b.emc, prec))) return rc;
  if ((rc = upload(s->qpar, &b.qpar, prec))) return rc;
  if (s->has_pcell && (rc = upload(s->pcell, &b.pcell, prec))) return rc;
  if (s->has_b2 && (rc = upload(s->pcell2, &b.pcell2, prec))) return rc;
  if (prec == 1) {
    // FP32 records of rho probes hold rho_ab - rho_ab(ref) (the constant term
    // is added in FP64 when the records are fetched), so that a population
    // near 1 keeps the full FP32 precision of its deviation
    std::vector<double> co = s->pr_coef;
    const int K = s->K;
    for (size_t k = 0; k < s->pr_cell.size(); ++k) co[k * (K + 1) + K] = 0.0;
    if ((rc = upload(co, &b.pr_coef, prec))) return rc;
  } else if ((rc = upload(s->pr_coef, &b.pr_coef, prec))) {
    return rc;
  }
  if (prec == 1 && !s->tcw.empty() && (rc = upload_raw(s->tcw, &b.tcw))) return rc;
  const size_t nrec = std::max<size_t>(1, s->pr_cell.size()) * (size_t)s->nt;
  if ((e = cudaMalloc(&b.rec, nrec * rb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc records");
  if ((e = cudaMemset(b.rec, 0, nrec * rb)) != cudaSuccess) return cuda_fail(e, "cudaMemset");
  for (auto &sr : s->src) {
    void *p = nullptr;
    if ((rc = upload_src(sr.sH, &p, prec))) return rc;
    b.src_tabs.push_back(p);
    if ((rc = upload_src(sr.sE, &p, prec))) return rc;
    b.src_tabs.push_back(p);
  }
  b.ready = true;
  return 0;
}

mbs::Args make_args(mbs_scenario_s *s, int prec) {
  Bundle &b = s->b[prec];
  mbs::Args a{};
  a.prec = prec;
  a.N = s->N;
  a.K = s->K;
  a.P = s->P;
  a.nx = s->dev->nx;
  a.ld = s->ld;
  a.off = s->off;
  a.nt = s->nt;
  for (int i = 0; i < 2; ++i) {
    a.E[i] = b.E[i];
    a.H[i] = b.H[i];
    a.El[i] = b.El[i];
    a.Hl[i] = b.Hl[i];
    a.D[i] = b.D[i];
    a.C[i] = b.C[i];
  }
  a.pd = b.pd;
  a.mat = s->d_mat;
  a.n_mat_all = (int)s->qslot.size();
  a.emc = b.emc;
  a.qslot = s->d_qslot;
  a.qpar = b.qpar;
  a.n_slot = s->n_slot;
  a.qstride = s->qstride;
  a.pcell = s->has_pcell ? b.pcell : nullptr;
  a.pcell2 = s->has_b2 ? b.pcell2 : nullptr;

  a.n_src = (int)s->src.size();
  for (size_t k = 0; k < s->src.size(); ++k) {
    a.src[k].kind = s->src[k].kind;
    a.src[k].face = s->src[k].face;
    a.src[k].cell = s->src[k].cell;
    a.src[k].sH = b.src_tabs[2 * k];
    a.src[k].sE = b.src_tabs[2 * k + 1];
  }
  a.bc_l = s->dev->bc_l;
  a.bc_r = s->dev->bc_r;
  a.r_l = s->dev->r_l;
  a.r_r = s->dev->r_r;
  a.bprev[0] = b.bprev[0];
  a.bprev[1] = b.bprev[1];
  a.kmur_l = s->kmur_l;
  a.kmur_r = s->kmur_r;
  a.n_probe = (int)s->pr_cell.size();
  a.pr_cell = s->d_pr_cell;
  a.pr_q = s->d_pr_q;
  a.pr_coef = b.pr_coef;
  a.tcw = b.tcw;
  a.rec = b.rec;
  a.zref = s->d_zref;
  a.flags = s->d_flags;
  return a;
}

void free_scenario(mbs_scenario_s *s) {
  for (auto &b : s->b) free_bundle(b);
  cudaFree(s->d_mat);
  cudaFree(s->d_qslot);
  cudaFree(s->d_pr_cell);
  cudaFree(s->d_pr_q);
  cudaFree(s->d_flags);
  cudaFree(s->d_chk_cells);
  cudaFree(s->d_zref);
  cudaFree(s->d_chk_min);
  cudaFree(s->d_chk_tr);
}

double light_speed(const MatDesc &m) { return 1.0 / std::sqrt(kEps0 * m.eps_r * kMu0 * m.mu_r); }

// source envelopes (Sec. 3.1.2, sech_pulse / gaussian_pulse) at x = (t - t0)/tau
double envelope(int shape, double x) { return shape == MBS_SHAPE_GAUSS ? std::exp(-x * x) : 1.0 / std::cosh(x); }

}  // namespace

int mbs::set_error(int code, const char *msg) { return fail(code, "%s", msg); }

// ============================================================ C ABI
extern "C" {

const char *mbs_last_error(void) { return g_err.c_str(); }

int mbs_abi_version(void) { return MBS_ABI_VERSION; }

int mbs_device_create(const mbs_qm_desc *qms, int n_qm, const mbs_material *mats, int n_mat,
                      const mbs_region *regions, int n_regions, double length, int n_cells, mbs_bc bc,
                      const double *per_cell_jitter, mbs_device_t *out) {
  g_err.clear();
  if (!out) return fail(MBS_E_INVALID, "out is NULL");
  *out = nullptr;
  if (n_qm < 0 || (n_qm > 0 && !qms)) return fail(MBS_E_INVALID, "bad quantum description list");
  if (n_mat < 1 || n_mat > 250 || !mats) return fail(MBS_E_INVALID, "need 1..250 materials");
  if (n_regions < 1 || !regions) return fail(MBS_E_INVALID, "need at least one region");
  if (!(length > 0) || n_cells < 8) return fail(MBS_E_INVALID, "need length > 0 and n_cells >= 8");
  if (n_cells > (1 << 30)) return fail(MBS_E_INVALID, "n_cells too large");
  // 0: absorbing (first-order Mur), 1: mirror, 2: partially reflecting
  auto refl = [](double r) { return r == 0.0 ? 0 : (r == 1.0 ? 1 : (r > 0.0 && r < 1.0 ? 2 : -1)); };
  if (refl(bc.refl_left) < 0 || refl(bc.refl_right) < 0)
    return fail(MBS_E_INVALID, "reflectivity must be in [0, 1]");
  auto dev = std::make_unique<mbs_device_s>();
  dev->nx = n_cells;
  dev->length = length;
  dev->dz = length / n_cells;
  dev->bc_l = refl(bc.refl_left);
  dev->bc_r = refl(bc.refl_right);
  dev->r_l = -std::sqrt(bc.refl_left);
  dev->r_r = -std::sqrt(bc.refl_right);
  int status = MBS_OK;
  for (int i = 0; i < n_qm; ++i) {
    QDesc q;
    const int rc = build_qdesc(qms[i], q);
    if (rc < 0) return rc;
    if (rc == MBS_W_NOT_PSD) status = MBS_W_NOT_PSD;
    dev->qms.push_back(std::move(q));
  }
  for (int i = 0; i < n_mat; ++i) {
    const mbs_material &m = mats[i];
    if (!(m.eps_r > 0) || !(m.mu_r > 0) || !(m.sigma >= 0) || !(m.overlap >= 0))
      return fail(MBS_E_INVALID, "material %d: need eps_r, mu_r > 0, sigma, overlap >= 0", i);
    if (m.qm < -1 || m.qm >= n_qm) return fail(MBS_E_INVALID, "material %d: bad quantum description index", i);
    dev->mats.push_back({m.eps_r, m.mu_r, m.sigma, m.overlap, m.qm});
  }
  for (int r = 0; r < n_regions; ++r)
    if (regions[r].material < 0 || regions[r].material >= n_mat)
      return fail(MBS_E_INVALID, "region %d: bad material index", r);
  dev->cell_mat.resize(n_cells);
  for (int m = 0; m < n_cells; ++m) {
    const double x = (m + 0.5) * dev->dz;
    int k = -1;
    for (int r = 0; r < n_regions; ++r)
      if (x >= regions[r].x_start && x < regions[r].x_end) {
        k = regions[r].material;
        break;
      }
    if (k < 0) return fail(MBS_E_INVALID, "cell %d (x = %g m) lies in no region", m, x);
    dev->cell_mat[m] = (uint8_t)k;
    const int q = dev->mats[k].qm;
    if (q >= 0) {
      if (dev->N == 0) dev->N = dev->qms[q].N;
      if (dev->qms[q].N != dev->N) return fail(MBS_E_INVALID, "media with different level counts in one device");
    }
  }
  if (per_cell_jitter) {
    dev->jitter.assign(per_cell_jitter, per_cell_jitter + (size_t)2 * n_cells);
    for (double v : dev->jitter)
      if (!std::isfinite(v) || v < 0) return fail(MBS_E_INVALID, "per-cell factors must be finite and >= 0");
  }
  *out = dev.release();
  return status;
}

void mbs_device_destroy(mbs_device_t d) { delete d; }

int mbs_device_propagators(mbs_device_t dev, int qm, double dt, double *lambda, double *V, double *A,
                           double *Ah, double *c, double *zref, double *g, double *g0) {
  g_err.clear();
  if (!dev || qm < 0 || qm >= (int)dev->qms.size() || !(dt > 0)) return fail(MBS_E_INVALID, "bad arguments");
  const QDesc &q = dev->qms[qm];
  const int N = q.N, N2 = N * N, K = N2 - 1;
  Step s;
  build_step(q, 1.0, dt, s);
  if (lambda) std::copy(q.lambda.begin(), q.lambda.end(), lambda);
  if (V)
    for (int i = 0; i < N2; ++i) {
      V[2 * i] = q.V[i].real();
      V[2 * i + 1] = q.V[i].imag();
    }
  if (A) std::copy(s.AK.begin(), s.AK.end(), A);
  if (Ah) std::copy(s.Ah.begin(), s.Ah.end(), Ah);
  if (c) std::copy(s.c.begin(), s.c.end(), c);
  if (zref) std::copy(q.yref.begin(), q.yref.end(), zref);
  if (g) std::copy(s.g.begin(), s.g.end(), g);
  if (g0) *g0 = s.g0;
  (void)K;
  return MBS_OK;
}

int mbs_scenario(mbs_device_t dev, double dt_or_0, double courant, double t_end, long long n_steps,
                 const mbs_source *src, int n_src, const mbs_probe *probes, int n_probes, mbs_scenario_t *out) {
  g_err.clear();
  if (!out) return fail(MBS_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!dev) return fail(MBS_E_INVALID, "device is NULL");
  if (n_src < 0 || n_src > mbs::MAXSRC || (n_src && !src)) return fail(MBS_E_INVALID, "0..%d sources", mbs::MAXSRC);
  if (n_probes < 0 || n_probes > mbs::MAXPROBE || (n_probes && !probes))
    return fail(MBS_E_INVALID, "0..%d probes", mbs::MAXPROBE);
  const int nx = dev->nx;
  const double dz = dev->dz;
  double cmax = 0;
  for (int m = 0; m < nx; ++m) cmax = std::max(cmax, light_speed(dev->mats[dev->cell_mat[m]]));
  double dt;
  if (dt_or_0 > 0) {
    dt = dt_or_0;
    if (dt > dz / cmax * (1 + 1e-12)) return fail(MBS_E_INVALID, "dt exceeds the Courant limit dz / c_max");
  } else {
    if (!(courant > 0 && courant <= 1)) return fail(MBS_E_INVALID, "courant must be in (0, 1]");
    dt = courant * dz / cmax;
  }
  long long nt = n_steps > 0 ? n_steps : (long long)std::ceil(t_end / dt);
  if (nt < 1) return fail(MBS_E_INVALID, "no time steps (t_end <= 0 and n_steps <= 0)");
  if (nt > (1LL << 31)) return fail(MBS_E_INVALID, "too many steps");

  auto s = std::make_unique<mbs_scenario_s>();
  s->dev = dev;
  s->dt = dt;
  s->nt = nt;
  const int N = std::max(dev->N, 2);
  s->N = N;
  s->K = N * N - 1;
  s->P = N * (N - 1) / 2;
  const int K = s->K, P = s->P, N2 = N * N;
  s->ld = ((nx + 2 * mbs::PAD) + 31) / 32 * 32;
  const int n_mat = (int)dev->mats.size();
  const double eta0 = std::sqrt(kMu0 / kEps0);

  // EM coefficients (normalised H^ = eta0 H); the extra last material is the
  // inert pad outside the domain
  s->emc.assign((size_t)(n_mat + 1) * 4, 0.0);
  for (int i = 0; i < n_mat; ++i) {
    const MatDesc &m = dev->mats[i];
    const double eps = kEps0 * m.eps_r, k = dt * m.sigma / (2 * eps);
    s->emc[i * 4 + 0] = (1 - k) / (1 + k) - 1.0;   // a' - 1 (exactly 0 without loss)
    s->emc[i * 4 + 1] = (dt / eps) / (1 + k) / (dz * eta0);
    s->emc[i * 4 + 2] = dt * eta0 / (dz * kMu0 * m.mu_r);
  }
  // slots: one per material with a quantum description
  s->qslot.assign(n_mat + 1, -1);
  std::vector<int> slot_mat;
  for (int i = 0; i < n_mat; ++i)
    if (dev->mats[i].qm >= 0) {
      s->qslot[i] = (int)slot_mat.size();
      slot_mat.push_back(i);
    }
  s->n_slot = (int)slot_mat.size();
  s->qstride = mbs::q_stride(N);
  s->qpar.assign((size_t)std::max(1, s->n_slot) * s->qstride, 0.0);
  s->zref.assign((size_t)std::max(1, s->n_slot) * N2, 0.0);
  std::vector<Step> steps(s->n_slot);
  for (int sl = 0; sl < s->n_slot; ++sl) {
    const MatDesc &m = dev->mats[slot_mat[sl]];
    const QDesc &q = dev->qms[m.qm];
    Step &st = steps[sl];
    build_step(q, 1.0, dt, st);
    const double bp = (dt / (kEps0 * m.eps_r)) / (1 + dt * m.sigma / (2 * kEps0 * m.eps_r));
    const double cpl = bp * m.overlap * q.n3d;
    double *blk = &s->qpar[(size_t)sl * s->qstride];
    for (int i = 0; i < K * K; ++i) blk[i] = st.AKm1[i];
    for (int i = 0; i < K; ++i) {
      blk[K * K + i] = st.c[i];
      blk[K * K + K + i] = cpl * st.g[i];
    }
    blk[K * K + 2 * K] = cpl * st.g0;
    int p = 0;
    for (int j = 0; j < N; ++j)
      for (int k = j + 1; k < N; ++k, ++p) {
        blk[K * K + 2 * K + 1 + p] = (q.lambda[j] - q.lambda[k]) * dt / kHbar;
        blk[K * K + 2 * K + 1 + P + 2 * p] = q.yref[N + 2 * p];
        blk[K * K + 2 * K + 1 + P + 2 * p + 1] = q.yref[N + 2 * p + 1];
      }
    std::copy(q.yref.begin(), q.yref.end(), &s->zref[(size_t)sl * N2]);
  }

  for (double v : s->qpar)
    if (!std::isfinite(v)) return fail(MBS_E_NUMERIC, "non-finite step operator (check H0, mu, rates and dt)");
  if (N >= 4 && s->n_slot == 1) {
    s->tcw.resize(mbs::tc_weight_table(N, s->qpar.data(), nullptr));
    mbs::tc_weight_table(N, s->qpar.data(), s->tcw.data());
  }

  // per-cell state and (jittered media) per-cell step operators
  const int ld = s->ld, off = s->off;
  s->Dinit.assign((size_t)K * ld, 0.0);
  s->has_pcell = !dev->jitter.empty() && s->n_slot > 0;
  if (s->has_pcell) s->pcell.assign((size_t)mbs::pc_rows(N) * ld, 0.0);
  std::vector<double> d0_slot((size_t)std::max(1, s->n_slot) * K, 0.0);
  for (int sl = 0; sl < s->n_slot; ++sl) {
    const QDesc &q = dev->qms[dev->mats[slot_mat[sl]].qm];
    // x^0 - yref = (exp(L0 dt/2) - I) yinit + (yinit - yref)
    std::vector<double> x0(N2, 0.0);
    for (int i = 0; i < N2; ++i)
      for (int j = 0; j < N2; ++j) x0[i] += steps[sl].Ehm1[i * N2 + j] * q.yinit[j];
    for (int i = 0; i < K; ++i) d0_slot[sl * K + i] = x0[full_of(N, i)] + (q.yinit[full_of(N, i)] - q.yref[full_of(N, i)]);
  }
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : bad)
  for (int m = 0; m < nx; ++m) {
    const int mt = dev->cell_mat[m];
    const int sl = s->qslot[mt];
    if (sl < 0) continue;
    if (!s->has_pcell) {
      for (int i = 0; i < K; ++i) s->Dinit[(size_t)i * ld + off + m] = d0_slot[sl * K + i];
      continue;
    }
    const MatDesc &mm = dev->mats[mt];
    const QDesc &q = dev->qms[mm.qm];
    const double fd = dev->jitter[2 * m], fh = dev->jitter[2 * m + 1];
    Step st;
    build_step(q, fh, dt, st);
    const double bp = (dt / (kEps0 * mm.eps_r)) / (1 + dt * mm.sigma / (2 * kEps0 * mm.eps_r));
    const double cpl = bp * mm.overlap * q.n3d * fd;
    const size_t col = (size_t)off + m;
    for (int i = 0; i < K * K; ++i) s->pcell[(size_t)i * ld + col] = st.AKm1[i];
    for (int i = 0; i < K; ++i) {
      s->pcell[(size_t)(K * K + i) * ld + col] = st.c[i];
      s->pcell[(size_t)(K * K + K + i) * ld + col] = cpl * st.g[i];
    }
    s->pcell[(size_t)(K * K + 2 * K) * ld + col] = cpl * st.g0;
    std::vector<double> x0(N2, 0.0);
    for (int i = 0; i < N2; ++i)
      for (int j = 0; j < N2; ++j) x0[i] += st.Ehm1[i * N2 + j] * q.yinit[j];
    for (int i = 0; i < K; ++i)
      s->Dinit[(size_t)i * ld + col] = x0[full_of(N, i)] + (q.yinit[full_of(N, i)] - q.yref[full_of(N, i)]);
    if (!std::isfinite(st.AK[0])) ++bad;
  }
  if (bad) return fail(MBS_E_NUMERIC, "non-finite per-cell propagator");

  // structured two-level rows: every medium cell's step operator has the
  // optical-Bloch pattern (A - I non-zero only at (0,0), (0,2), (1,1), (2,0),
  // (2,2); no affine offset; no coupling through component 1)
  if (N == 2 && s->n_slot > 0) {
    const int stride = s->qstride;
    auto val = [&](int m, int slot, int r) {   // dense row r of cell m
      return s->has_pcell ? s->pcell[(size_t)r * ld + off + m] : s->qpar[(size_t)slot * stride + r];
    };
    s->pcell2.assign((size_t)7 * ld, 0.0);
    int bad2 = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad2)
    for (int m = 0; m < nx; ++m) {
      const int sl = s->qslot[dev->cell_mat[m]];
      if (sl < 0) continue;
      double A[9], c[3], w[3];
      for (int r = 0; r < 9; ++r) A[r] = val(m, sl, r);
      for (int r = 0; r < 3; ++r) {
        c[r] = val(m, sl, 9 + r);
        w[r] = val(m, sl, 12 + r);
      }
      const double w0 = val(m, sl, 15);
      double amax = 0, wmax = 0;
      for (double x : A) amax = std::max(amax, std::fabs(x));
      for (double x : w) wmax = std::max(wmax, std::fabs(x));
      const double ta = 1e-13 * amax, tw = 1e-13 * wmax;
      if (std::fabs(A[1]) > ta || std::fabs(A[3]) > ta || std::fabs(A[5]) > ta || std::fabs(A[7]) > ta ||
          std::fabs(c[0]) > 1e-13 || std::fabs(c[1]) > 1e-13 || std::fabs(c[2]) > 1e-13 || std::fabs(w[1]) > tw ||
          std::fabs(w0) > tw) {
        ++bad2;
        continue;
      }
      const size_t col = (size_t)off + m;
      const double rows[7] = {A[0], A[2], A[4], A[6], A[8], w[0], w[2]};
      for (int r = 0; r < 7; ++r) s->pcell2[(size_t)r * ld + col] = rows[r];
    }
    s->has_b2 = bad2 == 0;
    if (!s->has_b2) s->pcell2.clear();
  }
  // sources
  for (int k = 0; k < n_src; ++k) {
    const mbs_source &sr = src[k];
    if (sr.kind < 0 || sr.kind > 2) return fail(MBS_E_INVALID, "source %d: bad kind", k);
    if (sr.shape != MBS_SHAPE_SECH && sr.shape != MBS_SHAPE_GAUSS) return fail(MBS_E_INVALID, "source %d: bad shape", k);
    if (sr.cell < 2 || sr.cell > nx - 3) return fail(MBS_E_INVALID, "source %d: cell must be in [2, n_cells-3]", k);
    if (!(sr.tau > 0)) return fail(MBS_E_INVALID, "source %d: tau must be > 0", k);
    if (!std::isfinite(sr.e0) || !std::isfinite(sr.tau) || !std::isfinite(sr.t0) || !std::isfinite(sr.omega) ||
        !std::isfinite(sr.phase))
      return fail(MBS_E_INVALID, "source %d: non-finite parameter", k);
    SrcHost h;
    h.kind = sr.kind;
    h.cell = sr.cell;
    h.face = sr.kind == MBS_SRC_TFSF_RIGHT ? sr.cell : (sr.kind == MBS_SRC_TFSF_LEFT ? sr.cell + 1 : -1);
    h.sH.assign(nt, 0.0);
    h.sE.assign(nt, 0.0);
    const MatDesc &ms = dev->mats[dev->cell_mat[sr.cell]];
    const double cs = light_speed(ms), eta_s = std::sqrt(kMu0 * ms.mu_r / (kEps0 * ms.eps_r));
    const double bh = s->emc[dev->cell_mat[sr.cell] * 4 + 1];
    const double ch = h.face >= 0 ? s->emc[dev->cell_mat[h.face] * 4 + 2] : 0.0;
    auto S = [&](double t) { return sr.e0 * envelope(sr.shape, (t - sr.t0) / sr.tau) * std::sin(sr.omega * t + sr.phase); };
    for (long long n = 0; n < nt; ++n) {
      const double tn = n * dt;
      if (sr.kind == MBS_SRC_HARD) {
        h.sE[n] = S(tn + dt);
      } else {
        h.sH[n] = (sr.kind == MBS_SRC_TFSF_RIGHT ? -1.0 : 1.0) * ch * S(tn);
        h.sE[n] = bh * (eta0 / eta_s) * S(tn + 0.5 * dt + 0.5 * dz / cs);
      }
    }
    s->src.push_back(std::move(h));
  }
  // boundaries
  {
    const double cl = light_speed(dev->mats[dev->cell_mat[0]]), cr = light_speed(dev->mats[dev->cell_mat[nx - 1]]);
    s->kmur_l = (cl * dt - dz) / (cl * dt + dz);
    s->kmur_r = (cr * dt - dz) / (cr * dt + dz);
  }
  // probes
  s->pr_coef.assign((size_t)std::max(1, n_probes) * (K + 1), 0.0);
  for (int k = 0; k < n_probes; ++k) {
    const mbs_probe &p = probes[k];
    if (p.cell < 0 || p.cell >= nx) return fail(MBS_E_INVALID, "probe %d: cell out of range", k);
    if (p.quantity < 0 || p.quantity > 3) return fail(MBS_E_INVALID, "probe %d: bad quantity", k);
    s->pr_cell.push_back(p.cell);
    s->pr_q.push_back(p.quantity);
    if (p.quantity >= 2) {
      const int mt = dev->cell_mat[p.cell], sl = s->qslot[mt];
      if (sl < 0) return fail(MBS_E_INVALID, "probe %d: density matrix requested in a cell without medium", k);
      if (p.i < 0 || p.j < 0 || p.i >= N || p.j >= N) return fail(MBS_E_INVALID, "probe %d: level index", k);
      const QDesc &q = dev->qms[dev->mats[mt].qm];
      Step st;
      build_step(q, dev->jitter.empty() ? 1.0 : dev->jitter[2 * p.cell + 1], dt, st);
      const std::vector<double> h = rho_functional(q, p.i, p.j, p.quantity == MBS_Q_RHO_IM);
      std::vector<double> hA(N2, 0.0);   // Ah^T h
      for (int c = 0; c < N2; ++c)
        for (int r = 0; r < N2; ++r) hA[c] += h[r] * st.Ah[r * N2 + c];
      double h0 = 0;
      for (int c = 0; c < N2; ++c) h0 += hA[c] * q.yref[c];
      double *co = &s->pr_coef[(size_t)k * (K + 1)];
      for (int i = 0; i < K; ++i) co[i] = hA[full_of(N, i)] - (i < N - 1 ? hA[N - 1] : 0.0);
      co[K] = h0;
    }
  }
  // cells for the state check: probes plus a strided sample of media
  {
    std::vector<int> med;
    for (int m = 0; m < nx; ++m)
      if (s->qslot[dev->cell_mat[m]] >= 0) med.push_back(m);
    const size_t want = 4096;
    const size_t stride = std::max<size_t>(1, med.size() / want);
    for (size_t i = 0; i < med.size(); i += stride) s->chk_cells.push_back(med[i]);
    for (int c : s->pr_cell) s->chk_cells.push_back(c);
  }

  // device-resident tables shared by both precisions
  cudaError_t e = cudaGetDevice(&s->device_id);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  g_h2d = &s->h2d_bytes;
  std::vector<uint8_t> matpad(ld, (uint8_t)n_mat);
  for (int m = 0; m < nx; ++m) matpad[off + m] = dev->cell_mat[m];
  int rc;
  if ((rc = upload_raw(matpad, &s->d_mat)) || (rc = upload_raw(s->qslot, &s->d_qslot)) ||
      (rc = upload_raw(s->pr_cell, &s->d_pr_cell)) || (rc = upload_raw(s->pr_q, &s->d_pr_q)) ||
      (rc = upload_raw(s->chk_cells, &s->d_chk_cells)) || (rc = upload_raw(s->zref, &s->d_zref))) {
    g_h2d = nullptr;
    free_scenario(s.get());
    return rc;
  }
  g_h2d = nullptr;
  const size_t nchk = std::max<size_t>(1, s->chk_cells.size());
  if ((e = cudaMalloc(&s->d_flags, 4 * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_chk_min, nchk * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_chk_tr, nchk * sizeof(double))) != cudaSuccess) {
    free_scenario(s.get());
    return cuda_fail(e, "cudaMalloc");
  }
  *out = s.release();
  return MBS_OK;
}

void mbs_scenario_destroy(mbs_scenario_t s) {
  if (!s) return;
  drop_graphs_of(s);
  free_scenario(s);
  delete s;
}

int mbs_scenario_info(mbs_scenario_t s, double *dt, double *dz, long long *n_steps) {
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (dt) *dt = s->dt;
  if (dz) *dz = s->dev->dz;
  if (n_steps) *n_steps = s->nt;
  return MBS_OK;
}

// Upload the precision's tables on first use and reset the state to the
// initial condition (all asynchronous on `st`).
static int prepare_solve(mbs_scenario_s *s, int prec, cudaStream_t st) {
  g_h2d = &s->h2d_bytes;
  int rc = ensure_bundle(s, prec);
  g_h2d = nullptr;
  if (rc) return rc;
  s->d2h_bytes = 0;
  s->launches = 0;
  Bundle &b = s->b[prec];
  const size_t row = (size_t)s->ld * b.rb;
  const int K = s->K;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    if ((e = cudaMemsetAsync(b.E[i], 0, row, st)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(b.H[i], 0, row, st)) != cudaSuccess) break;
    if (b.El[i] && (e = cudaMemsetAsync(b.El[i], 0, row, st)) != cudaSuccess) break;
    if (b.Hl[i] && (e = cudaMemsetAsync(b.Hl[i], 0, row, st)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(b.C[i], 0, row * K, st)) != cudaSuccess) break;
    e = cudaMemcpyAsync(b.D[i], b.Dinit, row * K, cudaMemcpyDeviceToDevice, st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b.pd, 0, row, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_flags, 0, 4 * sizeof(int), st);
  // the initial field E^0 (also E^{-1}: a static field before the first step)
  double eb[2] = {0.0, 0.0};
  if (e == cudaSuccess && !s->e_init.empty()) {
    const int nx = s->dev->nx;
    eb[0] = s->e_init[0];
    eb[1] = s->e_init[nx - 1];
    if (prec == 0) {
      for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync((double *)b.E[i] + s->off, s->e_init.data(), nx * sizeof(double), cudaMemcpyHostToDevice, st);
    } else {
      s->e_init_f.resize(2 * (size_t)nx);
      for (int m = 0; m < nx; ++m) {
        const float hi = (float)s->e_init[m];
        s->e_init_f[m] = hi;
        s->e_init_f[nx + m] = (float)(s->e_init[m] - (double)hi);
      }
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMemcpyAsync((float *)b.E[i] + s->off, s->e_init_f.data(), nx * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync((float *)b.El[i] + s->off, s->e_init_f.data() + nx, nx * sizeof(float),
                              cudaMemcpyHostToDevice, st);
      }
    }
  }
  if (e == cudaSuccess) {
    if (prec == 0) {
      s->bprev_init_d = {eb[0], 0.0, eb[1], 0.0};
      for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(b.bprev[i], s->bprev_init_d.data(), 4 * sizeof(double), cudaMemcpyHostToDevice, st);
    } else {
      const float l = (float)eb[0], r = (float)eb[1];
      s->bprev_init_f = {l, (float)(eb[0] - (double)l), r, (float)(eb[1] - (double)r)};
      for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(b.bprev[i], s->bprev_init_f.data(), 4 * sizeof(float), cudaMemcpyHostToDevice, st);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "state reset");
  return MBS_OK;
}

// Tile depth when the caller leaves it to the library: the fastest measured
// on GB300 (two levels: 24 steps, three levels: 32, tensor-core tiles: 8 for
// 128 cells, 20 for 256 cells).
static int default_tile_steps(int N, int tc_cells = 128) { return N == 2 ? 24 : N == 3 ? 32 : tc_cells == 256 ? 20 : 8; }

// Whether scenario s runs on the tensor-core tiles (N = 4..6 in FP32 with a
// single medium and no per-cell operators).
static bool uses_tc(const mbs_scenario_s *s, int prec) {
  return s->N >= 4 && mbs::tiled_tc_supported(prec, s->N) && s->n_slot == 1 && !s->has_pcell;
}

static int default_algo(const mbs_scenario_s *s, int prec) {
  if (uses_tc(s, prec)) return MBS_ALGO_TILED;
  return mbs::tiled_supported(prec, s->N) && (!s->has_pcell || s->N == 2) ? MBS_ALGO_TILED : MBS_ALGO_PLAIN;
}

// Whether the tiled kernels cover scenario s with tile depth T (sets the error).
static int tiled_ok(const mbs_scenario_s *s, int prec, int T) {
  if (s->N >= 4) {
    if (!uses_tc(s, prec))
      return fail(MBS_E_INVALID,
                  "tiled kernels for N >= 4 need FP32, one medium and no per-cell factors; use the plain algorithm");
    if (!mbs::tiled_tc_geometry_ok(s->dev->nx, s->tc_cells, T))
      return fail(MBS_E_INVALID,
                  "tile_steps %d does not fit %d-cell tensor-core tiles on this grid (1..20 always fit 128-cell tiles)",
                  T, s->tc_cells);
    return MBS_OK;
  }
  if (!mbs::tiled_supported(prec, s->N) || (s->has_pcell && s->N != 2))
    return fail(MBS_E_INVALID, "tiled kernels cover N = 2 (also with per-cell factors) and N = 3");
  const int R = mbs::tile_lane_cells(s->N);
  if (T % 4 != 0 || T < 4 || T > mbs::tile_max_steps(s->N))
    return fail(MBS_E_INVALID, "tile_steps must be a multiple of 4 in [4, %d]", mbs::tile_max_steps(s->N) / 4 * 4);
  // each lane's R-cell group must hold at most one medium material
  for (int g = 0; g * R < s->dev->nx; ++g) {
    int sl = -1;
    for (int j = 0; j < R && g * R + j < s->dev->nx; ++j) {
      const int q = s->qslot[s->dev->cell_mat[g * R + j]];
      if (q >= 0 && sl >= 0 && q != sl)
        return fail(MBS_E_INVALID, "two media meet inside a %d-cell group; use the plain algorithm", R);
      if (q >= 0) sl = q;
    }
  }
  return MBS_OK;
}

static int launch_state_check(mbs_scenario_s *s, const mbs::Args &a, int c, cudaStream_t st) {
  const int nchk = (int)s->chk_cells.size();
  if (!nchk) return 0;
  ++s->launches;
  return mbs::launch_check(a, c, s->d_chk_cells, nchk, s->d_chk_min, s->d_chk_tr, s->d_zref, nullptr, st);
}

// The periodic check of Sec. 2.2's density-matrix properties at a step
// boundary: the sampled eigenvalue check, then the sweep over every cell
// (finiteness, populations and 2 x 2 minors; the FP32 Kahan fold).  With
// `wait` the host reads the status at once and returns true if it failed,
// so that the caller stops issuing launches; either way a failed check makes
// every later step launch of the scenario return at once.
static int periodic_check(mbs_scenario_s *s, const mbs::Args &a, int dcur, int ecur, int hcur, cudaStream_t st,
                          bool wait, bool *failed) {
  int r = launch_state_check(s, a, dcur, st);
  if (!r) {
    ++s->launches;
    r = mbs::launch_sweep(a, dcur, ecur, hcur, mbs::EIG_TOL, st);
  }
  if (r) return cuda_fail((cudaError_t)r, "check launch");
  *failed = false;
  if (wait) {
    int flags[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(flags, s->d_flags, sizeof flags, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "check status");
    s->d2h_bytes += sizeof flags;
    *failed = flags[0] != 0 || flags[1] != 0;
  }
  return MBS_OK;
}

// After the stream has drained: read the check results and device flags.
static int finish_solve(mbs_scenario_s *s, int prec, int cur, long long steps_run = -1) {
  cudaError_t e;
  s->solved_prec = prec;
  s->last_cur = cur;
  s->steps_run = steps_run < 0 ? s->nt : steps_run;
  const int nchk = (int)s->chk_cells.size();
  int flags[4] = {0, 0, 0, 0};
  if ((e = cudaMemcpy(flags, s->d_flags, sizeof flags, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "flags");
  s->d2h_bytes += sizeof flags + (long long)nchk * 2 * sizeof(double);
  s->st_min = 1e300;
  s->st_trace = 0;
  if (nchk) {
    std::vector<double> mn(nchk), tr(nchk);
    if ((e = cudaMemcpy(mn.data(), s->d_chk_min, nchk * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(tr.data(), s->d_chk_tr, nchk * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "check results");
    for (int i = 0; i < nchk; ++i) {
      s->st_min = std::min(s->st_min, mn[i]);
      s->st_trace = std::max(s->st_trace, tr[i]);
    }
  } else {
    s->st_min = 0;
  }
  if (flags[1]) return fail(MBS_E_TIMEOUT, "a bounded wait on the tensor cores gave up");
  if (flags[0] & 1) return fail(MBS_E_NUMERIC, "non-finite state after %lld steps", s->steps_run);
  if (flags[0]) return fail(MBS_E_NUMERIC, "density matrix not positive semidefinite after %lld steps", s->steps_run);
  if (nchk && s->st_min < -1e-6) return fail(MBS_E_NUMERIC, "density matrix eigenvalue %.3g < -1e-6", s->st_min);
  return MBS_OK;
}

}  // extern "C"

// ------------------------------------------------------------ autotuning
// Tile depth by measurement: every candidate depth runs one warm-up launch and
// two timed rounds of three launches (CUDA events on the solve stream) of the
// scenario (or of the whole batch group) from its current state; the faster
// round counts and the fastest time per step wins.  The caller resets the state afterwards.  Results are cached for the
// process, keyed by level count, precision, kernel variant and the cell and
// step counts, so a workload shape is tuned once.
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;

static std::vector<int> tile_candidates(int N, long long nt) {
  std::vector<int> c = N >= 4 ? std::vector<int>{6, 8, 10, 12, 14, 16, 20}
                     : N == 3 ? std::vector<int>{16, 20, 24, 28, 32, 40, 48}
                              : std::vector<int>{12, 16, 20, 24, 28, 32, 40, 48};
  std::vector<int> out;
  for (int T : c)
    if (T <= nt) out.push_back(T);
  return out;
}

static int tiled_launch(const mbs_scenario_s *s, const mbs::Args &a, long long n0, int ns, int T, int cur,
                        cudaStream_t st) {
  return s->N >= 4 ? mbs::launch_tiled_tc(a, s->tc_cells, n0, ns, T, cur, st)
                   : mbs::launch_tiled(a, n0, ns, T, cur, st);
}

// Candidate codes: the tile depth, plus 1000 for 256-cell tensor-core tiles.
static int code_steps(int code) { return code % 1000; }
static int code_cells(int code) { return code >= 1000 ? 256 : 128; }

// time `run(code, cur)` (which enqueues one launch) for every candidate; -1
// on error
template <class Run>
static int tune_loop(const std::vector<int> &cands, cudaStream_t st, Run run) {
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

// returns the winning candidate code (see code_steps / code_cells)
static int autotune_one(mbs_scenario_s *s, int prec, const mbs::Args &a, cudaStream_t st) {
  char key[128];
  std::snprintf(key, sizeof key, "1:%d:%d:%d:%d:%d", s->N, prec, s->N >= 4 ? 9 : mbs::tiled_variant(a), s->dev->nx,
                (int)std::min<long long>(s->nt, 1 << 30));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  std::vector<int> cands;
  for (int T : tile_candidates(s->N, s->nt)) {
    if (s->N < 4) {
      if (T <= mbs::tile_max_steps(s->N)) cands.push_back(T);
      continue;
    }
    if (mbs::tiled_tc_geometry_ok(s->dev->nx, 128, T)) cands.push_back(T);
  }
  if (s->N >= 4)
    for (int T : {12, 16, 20, 24, 32, 40})
      if (T <= s->nt && mbs::tiled_tc_geometry_ok(s->dev->nx, 256, T)) cands.push_back(1000 + T);
  if (cands.size() < 2) return default_tile_steps(s->N);
  const int saved = s->tc_cells;
  const int T = tune_loop(cands, st, [&](int c, int cur) {
    s->tc_cells = code_cells(c);
    return tiled_launch(s, a, 0, code_steps(c), code_steps(c), cur, st);
  });
  s->tc_cells = saved;
  if (T < 0) return default_tile_steps(s->N);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = T;
  return T;
}

static int solve_one(mbs_scenario_s *s, const mbs_opts &o, cudaStream_t st) {
  const int prec = o.precision;
  int rc = prepare_solve(s, prec, st);
  if (rc) return rc;
  mbs::Args a = make_args(s, prec);
  int algo = o.algo == MBS_ALGO_AUTO ? default_algo(s, prec) : o.algo;
  s->tc_cells = (o.flags & MBS_SOLVE_WIDE_TILES) ? 256 : 128;
  a.test_stall = (o.flags & MBS_SOLVE_TEST_STALL) ? 1 : 0;
  int T = o.tile_steps > 0 ? o.tile_steps : default_tile_steps(s->N, s->tc_cells);
  const int chk = o.check_every > 0 ? o.check_every : 0;
  int cur = 0;
  long long done = 0;
  bool stopped = false;   // a periodic check failed
  if (algo == MBS_ALGO_TILED) {
    if ((rc = tiled_ok(s, prec, T))) return rc;
    if (o.tile_steps <= 0 && (o.flags & MBS_SOLVE_AUTOTUNE)) {
      const int code = autotune_one(s, prec, a, st);
      T = code_steps(code);
      if (s->N >= 4) s->tc_cells = code_cells(code);
      if ((rc = prepare_solve(s, prec, st))) return rc;   // the trials advanced the state
    }
    while (done < s->nt && !stopped) {
      const int ns = (int)std::min<long long>(T, s->nt - done);
      int r = tiled_launch(s, a, done, ns, T, cur, st);
      ++s->launches;
      if (r) return cuda_fail((cudaError_t)r, "tiled launch");
      cur ^= 1;
      done += ns;
      if (chk && done < s->nt && (done / chk) != ((done - ns) / chk))
        if ((r = periodic_check(s, a, cur, cur, cur, st, true, &stopped))) return r;
    }
    s->tile_used = T;
  } else {
    for (long long n = 0; n < s->nt && !stopped; ++n) {
      int r = mbs::launch_plain_step(a, n, cur, st);
      s->launches += 2;
      if (r) return cuda_fail((cudaError_t)r, "plain launch");
      cur ^= 1;
      done = n + 1;
      if (chk && (n + 1) % chk == 0 && n + 1 < s->nt)   // plain: D, H in buffers 0, E in cur
        if ((r = periodic_check(s, a, 0, cur, 0, st, true, &stopped))) return r;
    }
    s->tile_used = 0;
  }
  // plain: D, H live in buffer 0, E in `cur`; tiled: everything in `cur`
  const int dcur = algo == MBS_ALGO_TILED ? cur : 0;
  if ((rc = launch_state_check(s, a, dcur, st))) return cuda_fail((cudaError_t)rc, "check launch");
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "solve");
  return finish_solve(s, prec, cur, done);
}

// Batched tiled solve: every round launches, per kernel variant, one grid
// over the blocks of all simulations still running, advancing them T steps.
// Blocks are ordered by their simulation's step count (longest first), so
// the running ones form a prefix and the grid shrinks as simulations end.
struct BatchGroup {
  int N, pm, T;
  std::vector<int> sims;   // indices into the batch, longest first
  std::vector<int2> tasks;
  std::vector<long long> task_nt;
  int max_mat = 0, max_slot = 0, max_stride = 0;
};

static void group_tasks(BatchGroup &g, const std::vector<mbs_scenario_s *> &ss, int T,
                        std::vector<int2> &tasks, std::vector<long long> &task_nt) {
  tasks.clear();
  task_nt.clear();
  const int own = mbs::tile_own(g.N, T);
  for (int i : g.sims) {
    const int n_tiles = (ss[i]->dev->nx + own - 1) / own;
    for (int w = 0; w < n_tiles; ++w) {
      tasks.push_back(make_int2(i, w));
      task_nt.push_back(ss[i]->nt);
    }
  }
}

// A batched solve recorded as a CUDA graph (MBS_SOLVE_GRAPH), with the device
// tables its launches read; replayed while the same scenarios are solved with
// the same options.  Destroying a member scenario drops the graph.
struct BatchGraph {
  std::vector<mbs_scenario_s *> members;
  int prec = 0, tile = 0, flags = 0, check_every = 0;
  std::vector<int> Ts;      // tile depth per group
  std::vector<int> sim_T;   // tile depth per member
  cudaGraphExec_t exec = nullptr;
  mbs::Args *d_args = nullptr;
  std::vector<int2 *> d_tasks;
};
static std::mutex g_graph_mu;
static std::vector<BatchGraph *> g_graphs;

static void free_graph(BatchGraph *g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  cudaFree(g->d_args);
  for (auto *p : g->d_tasks) cudaFree(p);
  delete g;
}

static void drop_graphs_of(mbs_scenario_s *s) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (size_t k = 0; k < g_graphs.size();) {
    auto &m = g_graphs[k]->members;
    if (std::find(m.begin(), m.end(), s) != m.end()) {
      free_graph(g_graphs[k]);
      g_graphs.erase(g_graphs.begin() + k);
    } else {
      ++k;
    }
  }
}

static int solve_batch(std::vector<mbs_scenario_s *> &ss, const mbs_opts &o, cudaStream_t st) {
  const int prec = o.precision;
  const int chk = o.check_every > 0 ? o.check_every : 0;
  int rc;
  for (auto *s : ss) {
    if ((rc = prepare_solve(s, prec, st))) return rc;
    if ((rc = tiled_ok(s, prec, o.tile_steps > 0 ? o.tile_steps : default_tile_steps(s->N)))) return rc;
  }
  // graphs need a stream that can be captured (not the legacy default stream)
  const bool use_graph = (o.flags & MBS_SOLVE_GRAPH) != 0 && st != nullptr;
  // replay a recorded graph of this very batch
  if (use_graph) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto *g : g_graphs)
      if (g->members == ss && g->prec == prec && g->tile == o.tile_steps && g->flags == o.flags &&
          g->check_every == chk) {
        cudaError_t e = cudaGraphLaunch(g->exec, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "batched graph replay");
        int status = MBS_OK;
        for (size_t i = 0; i < ss.size(); ++i) {
          const int T = g->sim_T[i];
          const long long rounds = (ss[i]->nt + T - 1) / T;
          ss[i]->launches = rounds;
          ss[i]->tile_used = T;
          rc = finish_solve(ss[i], prec, (int)(rounds % 2));
          if (rc && status == MBS_OK) status = rc;
        }
        return status;
      }
  }
  std::vector<BatchGroup> groups;
  std::vector<mbs::Args> args(ss.size());
  for (size_t i = 0; i < ss.size(); ++i) {
    args[i] = make_args(ss[i], prec);
    const int pm = mbs::tiled_variant(args[i]);
    if (pm < 0) return fail(MBS_E_INVALID, "scenario %zu is not covered by the tiled kernels", i);
    BatchGroup *g = nullptr;
    for (auto &x : groups)
      if (x.N == ss[i]->N && x.pm == pm) g = &x;
    if (!g) {
      groups.push_back(BatchGroup{ss[i]->N, pm, o.tile_steps > 0 ? o.tile_steps : default_tile_steps(ss[i]->N)});
      g = &groups.back();
    }
    g->sims.push_back((int)i);
    g->max_mat = std::max(g->max_mat, args[i].n_mat_all);
    g->max_slot = std::max(g->max_slot, args[i].n_slot);
    g->max_stride = std::max(g->max_stride, args[i].qstride);
  }
  for (auto &g : groups)
    std::stable_sort(g.sims.begin(), g.sims.end(), [&](int x, int y) { return ss[x]->nt > ss[y]->nt; });
  // device copy of the per-simulation arguments
  mbs::Args *d_args = nullptr;
  std::vector<int2 *> d_tasks(groups.size(), nullptr);
  auto cleanup = [&]() {
    cudaFree(d_args);
    for (auto *p : d_tasks) cudaFree(p);
  };
  cudaError_t e = cudaMalloc(&d_args, args.size() * sizeof(mbs::Args));
  if (e == cudaSuccess) e = cudaMemcpy(d_args, args.data(), args.size() * sizeof(mbs::Args), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "batch tables");
  }
  // tile depth per group: given, default, or measured
  if (o.tile_steps <= 0 && (o.flags & MBS_SOLVE_AUTOTUNE)) {
    for (auto &g : groups) {
      long long nt_min = LLONG_MAX, cells = 0, steps = 0;
      for (int i : g.sims) {
        nt_min = std::min(nt_min, ss[i]->nt);
        cells += ss[i]->dev->nx;
        steps += ss[i]->nt;
      }
      char key[160];
      std::snprintf(key, sizeof key, "B:%d:%d:%d:%zu:%lld:%lld", g.N, prec, g.pm, g.sims.size(), cells, steps);
      int T = -1;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) T = it->second;
      }
      if (T < 0) {
        std::vector<int> cands;
        for (int t : tile_candidates(g.N, nt_min))
          if (t <= mbs::tile_max_steps(g.N)) cands.push_back(t);
        const size_t smem = mbs::tiled_batch_smem(prec, g.N, g.max_mat, g.max_slot, g.max_stride);
        std::vector<int2> tk;
        std::vector<long long> tn;
        int2 *d_tk = nullptr;
        int last_T = -1;
        T = tune_loop(cands, st, [&](int t, int cur) {
          if (t != last_T) {   // tasks of this depth
            if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
            cudaFree(d_tk);
            d_tk = nullptr;
            group_tasks(g, ss, t, tk, tn);
            if (cudaMalloc(&d_tk, tk.size() * sizeof(int2)) != cudaSuccess ||
                cudaMemcpy(d_tk, tk.data(), tk.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
              return -1;
            last_T = t;
          }
          return mbs::launch_tiled_batch(prec, g.N, g.pm, d_args, d_tk, (int)tk.size(), smem, 0, t, cur, st);
        });
        cudaStreamSynchronize(st);
        cudaFree(d_tk);
        if (T < 0) T = default_tile_steps(g.N);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = T;
      }
      g.T = T;
    }
    for (auto *s : ss)   // the trials advanced the state
      if ((rc = prepare_solve(s, prec, st))) {
        cleanup();
        return rc;
      }
  }
  for (size_t k = 0; k < groups.size() && e == cudaSuccess; ++k) {
    group_tasks(groups[k], ss, groups[k].T, groups[k].tasks, groups[k].task_nt);
    e = cudaMalloc(&d_tasks[k], groups[k].tasks.size() * sizeof(int2));
    if (e == cudaSuccess)
      e = cudaMemcpy(d_tasks[k], groups[k].tasks.data(), groups[k].tasks.size() * sizeof(int2),
                     cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "batch tables");
  }
  std::vector<int> sim_T(ss.size());
  for (const auto &g : groups)
    for (int i : g.sims) sim_T[i] = g.T;
  // Each group runs on a stream of its own, forked from and joined back into
  // the caller's stream, so that one group's last, thinly populated rounds
  // overlap the other group's work.
  const size_t n_fork = groups.size() > 1 ? groups.size() : 0;
  std::vector<cudaStream_t> gst(groups.size(), st);
  std::vector<cudaEvent_t> ev(n_fork + 1, nullptr);
  auto release = [&]() {
    for (size_t k = 0; k < n_fork; ++k)
      if (gst[k] != st) cudaStreamDestroy(gst[k]);
    for (auto x : ev)
      if (x) cudaEventDestroy(x);
  };
  for (size_t k = 0; k < n_fork && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&gst[k], cudaStreamNonBlocking);
    if (e != cudaSuccess) gst[k] = st;
  }
  for (size_t k = 0; k < ev.size() && n_fork && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    release();
    cleanup();
    return cuda_fail(e, "batch streams");
  }
  // the launch sequence: fork, every group's rounds, join, per-simulation checks
  auto enqueue = [&]() -> int {
    cudaError_t x = cudaSuccess;
    if (n_fork) x = cudaEventRecord(ev[n_fork], st);
    for (size_t k = 0; k < n_fork && x == cudaSuccess; ++k) x = cudaStreamWaitEvent(gst[k], ev[n_fork], 0);
    if (x != cudaSuccess) return cuda_fail(x, "batch streams");
    for (size_t k = 0; k < groups.size(); ++k) {
      const auto &g = groups[k];
      const size_t smem = mbs::tiled_batch_smem(prec, g.N, g.max_mat, g.max_slot, g.max_stride);
      const long long nt_max = g.task_nt.front();
      int cur = 0;
      for (long long n0 = 0; n0 < nt_max; n0 += g.T) {
        // running blocks: a prefix of the tasks (sorted by step count)
        const int active = (int)(std::upper_bound(g.task_nt.begin(), g.task_nt.end(), n0,
                                                  [](long long v, long long y) { return v > y; }) -
                                 g.task_nt.begin());
        int r = mbs::launch_tiled_batch(prec, g.N, g.pm, d_args, d_tasks[k], active, smem, n0, g.T, cur, gst[k]);
        if (r) return cuda_fail((cudaError_t)r, "batched tiled launch");
        cur ^= 1;
        // periodic check: the sweep over every cell of the simulations that
        // ran this round (a failure stops that simulation's later rounds on
        // the device; the status is read when the batch has finished)
        const long long n1 = n0 + g.T;
        if (chk && n1 < nt_max && n1 / chk != n0 / chk) {
          r = mbs::launch_sweep_batch(prec, g.N, d_args, d_tasks[k], active, mbs::tile_own(g.N, g.T), n0, cur,
                                      mbs::EIG_TOL, gst[k]);
          if (r) return cuda_fail((cudaError_t)r, "batched sweep launch");
        }
      }
    }
    for (size_t k = 0; k < n_fork && x == cudaSuccess; ++k) {
      x = cudaEventRecord(ev[k], gst[k]);
      if (x == cudaSuccess) x = cudaStreamWaitEvent(st, ev[k], 0);
    }
    if (x != cudaSuccess) return cuda_fail(x, "batch streams");
    for (size_t i = 0; i < ss.size(); ++i) {
      const long long rounds = (ss[i]->nt + sim_T[i] - 1) / sim_T[i];
      const int r = launch_state_check(ss[i], args[i], (int)(rounds % 2), st);
      if (r) return cuda_fail((cudaError_t)r, "check launch");
    }
    return MBS_OK;
  };
  BatchGraph *graph = nullptr;
  if (use_graph) {
    cudaGraph_t gr = nullptr;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      release();
      cleanup();
      return cuda_fail(e, "graph capture (a NULL or legacy stream cannot be captured)");
    }
    rc = enqueue();
    const cudaError_t e2 = cudaStreamEndCapture(st, &gr);
    if (rc == MBS_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "graph capture");
    graph = new BatchGraph;
    if (rc == MBS_OK && (e = cudaGraphInstantiate(&graph->exec, gr, 0)) != cudaSuccess)
      rc = cuda_fail(e, "graph instantiation");
    if (gr) cudaGraphDestroy(gr);
    if (rc == MBS_OK && (e = cudaGraphLaunch(graph->exec, st)) != cudaSuccess) rc = cuda_fail(e, "graph launch");
    if (rc != MBS_OK) {
      free_graph(graph);
      release();
      cleanup();
      return rc;
    }
  } else {
    rc = enqueue();
    if (rc != MBS_OK) {
      cudaStreamSynchronize(st);
      release();
      cleanup();
      return rc;
    }
  }
  e = cudaStreamSynchronize(st);
  release();
  if (graph) {   // the graph keeps the tables it reads
    graph->members = ss;
    graph->prec = prec;
    graph->tile = o.tile_steps;
    graph->flags = o.flags;
    graph->check_every = chk;
    for (const auto &g : groups) graph->Ts.push_back(g.T);
    graph->sim_T = sim_T;
    graph->d_args = d_args;
    graph->d_tasks = d_tasks;
    std::lock_guard<std::mutex> lk(g_graph_mu);
    g_graphs.push_back(graph);
  } else {
    cleanup();
  }
  if (e != cudaSuccess) return cuda_fail(e, "batched solve");
  int status = MBS_OK;
  for (size_t i = 0; i < ss.size(); ++i) {
    auto *s = ss[i];
    const long long rounds = (s->nt + sim_T[i] - 1) / sim_T[i];
    s->launches = rounds;
    s->tile_used = sim_T[i];
    rc = finish_solve(s, prec, (int)(rounds % 2));
    if (rc && status == MBS_OK) status = rc;
  }
  return status;
}

extern "C" {

int mbs_solve(mbs_scenario_t *batch, int n_scen, const mbs_opts *opts, void *cuda_stream) {
  g_err.clear();
  if (!batch || n_scen < 1) return fail(MBS_E_INVALID, "empty batch");
  mbs_opts o{MBS_PREC_FP32, MBS_ALGO_AUTO, 0, 0, 0};
  if (opts) o = *opts;
  if (o.precision != MBS_PREC_FP64 && o.precision != MBS_PREC_FP32) return fail(MBS_E_INVALID, "bad precision");
  if (o.algo < 0 || o.algo > 2) return fail(MBS_E_INVALID, "bad algorithm");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  for (int i = 0; i < n_scen; ++i)
    if (!batch[i]) return fail(MBS_E_INVALID, "scenario %d is NULL", i);
  // several scenarios on the tiled path advance together, unless asked not to
  bool batched = n_scen > 1 && !(o.flags & MBS_SOLVE_ONE_AT_A_TIME) && o.algo != MBS_ALGO_PLAIN;
  for (int i = 0; i < n_scen && batched; ++i)
    batched = batch[i]->N <= 3 && default_algo(batch[i], o.precision) == MBS_ALGO_TILED;
  if (batched) {
    std::vector<mbs_scenario_s *> ss(batch, batch + n_scen);
    return solve_batch(ss, o, st);
  }
  for (int i = 0; i < n_scen; ++i) {
    const int rc = solve_one(batch[i], o, st);
    if (rc) return rc;
  }
  return MBS_OK;
}

int mbs_fetch_records(mbs_scenario_t s, int probe, double *out, size_t cap, size_t *n_written) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (probe < 0 || probe >= (int)s->pr_cell.size()) return fail(MBS_E_INVALID, "probe index out of range");
  const size_t n = (size_t)s->nt;
  if (n_written) *n_written = n;
  if (!out) return MBS_OK;
  if (cap < n) return fail(MBS_E_INVALID, "capacity %zu < %zu", cap, n);
  if (s->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  const Bundle &b = s->b[s->solved_prec];
  const double scale = s->pr_q[probe] == MBS_Q_H ? 1.0 / std::sqrt(kMu0 / kEps0) : 1.0;
  cudaError_t e;
  if (s->solved_prec == 0) {
    e = cudaMemcpy(out, (const double *)b.rec + (size_t)probe * n, n * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "fetch");
    s->d2h_bytes += (long long)(n * sizeof(double));
    if (scale != 1.0)
      for (size_t i = 0; i < n; ++i) out[i] *= scale;
  } else {
    std::vector<float> f(n);
    e = cudaMemcpy(f.data(), (const float *)b.rec + (size_t)probe * n, n * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "fetch");
    s->d2h_bytes += (long long)(n * sizeof(float));
    // rho probes: the FP32 record is the deviation from the reference value
    const double base = s->pr_q[probe] >= MBS_Q_RHO_RE ? s->pr_coef[(size_t)probe * (s->K + 1) + s->K] : 0.0;
    for (size_t i = 0; i < n; ++i) out[i] = scale * (double)f[i] + base;
  }
  return MBS_OK;
}

int mbs_scenario_set_field(mbs_scenario_t s, const double *e0, size_t n) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (!e0) {
    s->e_init.clear();
    return MBS_OK;
  }
  if (n != (size_t)s->dev->nx) return fail(MBS_E_INVALID, "the initial field needs n_cells = %d values", s->dev->nx);
  for (size_t m = 0; m < n; ++m)
    if (!std::isfinite(e0[m])) return fail(MBS_E_INVALID, "non-finite initial field at cell %zu", m);
  s->e_init.assign(e0, e0 + n);
  return MBS_OK;
}

int mbs_scenario_tile(mbs_scenario_t s, int *tile_steps) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (s->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  if (tile_steps) *tile_steps = s->tile_used;
  return MBS_OK;
}

int mbs_tile_plan(int n_levels, int tile_cells, int nx, int tile_steps, int *n_tiles) {
  g_err.clear();
  const int T = tile_steps;
  if (n_levels < 2 || n_levels > mbs::NMAX) return fail(MBS_E_INVALID, "n_levels %d outside [2, %d]", n_levels, mbs::NMAX);
  if (nx < 8) return fail(MBS_E_INVALID, "nx must be at least 8");
  if (n_levels >= 4) {
    if (!mbs::tiled_tc_geometry_ok(nx, tile_cells, T))
      return fail(MBS_E_INVALID, "tile_steps %d does not fit %d-cell tensor-core tiles on a %d-cell grid", T,
                  tile_cells, nx);
  } else {
    if (tile_cells != 32 * mbs::tile_warps(n_levels) * mbs::tile_lane_cells(n_levels))
      return fail(MBS_E_INVALID, "tiles of N = %d levels hold %d cells", n_levels,
                  32 * mbs::tile_warps(n_levels) * mbs::tile_lane_cells(n_levels));
    if (T % 4 != 0 || T < 4 || T > mbs::tile_max_steps(n_levels))
      return fail(MBS_E_INVALID, "tile_steps must be a multiple of 4 in [4, %d]", mbs::tile_max_steps(n_levels) / 4 * 4);
  }
  const int own = tile_cells - 2 * T;
  if (n_tiles) *n_tiles = (nx + own - 1) / own;
  return MBS_OK;
}

int mbs_scenario_tile_cells(mbs_scenario_t s, int *tile_cells) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (s->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  if (tile_cells)
    *tile_cells = s->tile_used == 0 ? 0 : s->N >= 4 ? s->tc_cells : 32 * mbs::tile_warps(s->N) * mbs::tile_lane_cells(s->N);
  return MBS_OK;
}

int mbs_scenario_counters(mbs_scenario_t s, long long *h2d_bytes, long long *d2h_bytes, long long *kernel_launches) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (h2d_bytes) *h2d_bytes = s->h2d_bytes;
  if (d2h_bytes) *d2h_bytes = s->d2h_bytes;
  if (kernel_launches) *kernel_launches = s->launches;
  return MBS_OK;
}

int mbs_scenario_stats(mbs_scenario_t s, double *max_trace_dev, double *min_eig, long long *n_steps) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (s->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  if (max_trace_dev) *max_trace_dev = s->st_trace;
  if (min_eig) *min_eig = s->st_min;
  if (n_steps) *n_steps = s->steps_run;
  return MBS_OK;
}

}  // extern "C"

// ============================================================ driven cells
// Batched single-cell Lindblad solver (include/mbs.h, mbs_cells_*): Nx = 1,
// the master equation of each system under its prescribed field.
struct mbs_cells_s {
  int N = 0, K = 0, P = 0, n_sys = 0, every = 1, rows = 0, n_tab = 0;
  double dt = 0;
  long long nt = 0, n_rec = 0;
  std::vector<double> prm, amp, tab, zref, Dinit;   // FP64 master copies
  std::vector<int> tab_id;
  struct Dev {
    bool ready = false;
    void *prm = nullptr, *D = nullptr, *C = nullptr, *amp = nullptr, *tab = nullptr, *rec = nullptr;
  } b[2];
  int *d_tab_id = nullptr, *d_flags = nullptr;
  double *d_zref = nullptr, *d_min = nullptr, *d_tr = nullptr;
  int solved_prec = -1;
  double st_min = 0, st_trace = 0;
};

namespace {

void free_cells(mbs_cells_s *c) {
  for (auto &b : c->b) {
    cudaFree(b.prm);
    cudaFree(b.D);
    cudaFree(b.C);
    cudaFree(b.amp);
    cudaFree(b.tab);
    cudaFree(b.rec);
    b = mbs_cells_s::Dev();
  }
  cudaFree(c->d_tab_id);
  cudaFree(c->d_flags);
  cudaFree(c->d_zref);
  cudaFree(c->d_min);
  cudaFree(c->d_tr);
}

int cells_device(mbs_cells_s *c, int prec) {
  auto &b = c->b[prec];
  if (!b.ready) {
    const size_t rb = rsize(prec), ns = (size_t)c->n_sys;
    int rc;
    if ((rc = upload(c->prm, &b.prm, prec)) || (rc = upload(c->amp, &b.amp, prec))) return rc;
    cudaError_t e = cudaMalloc(&b.D, ns * c->K * rb);
    if (e == cudaSuccess) e = cudaMalloc(&b.C, ns * c->K * rb);
    if (e == cudaSuccess) e = cudaMalloc(&b.rec, std::max<size_t>(1, (size_t)c->n_rec * c->N * ns) * rb);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (cells)");
    if (prec == 0) {
      if ((rc = upload(c->tab, &b.tab, 0))) return rc;
    } else {   // [n_tab][2][nt]: high words, then low words of each shape
      std::vector<float> f(2 * c->tab.size());
      for (int t = 0; t < c->n_tab; ++t)
        for (long long n = 0; n < c->nt; ++n) {
          const double v = c->tab[(size_t)t * c->nt + n];
          const float hi = (float)v;
          f[(size_t)t * 2 * c->nt + n] = hi;
          f[(size_t)t * 2 * c->nt + c->nt + n] = (float)(v - (double)hi);
        }
      if ((e = cudaMalloc(&b.tab, f.size() * sizeof(float))) != cudaSuccess ||
          (e = cudaMemcpy(b.tab, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "drive tables");
    }
    b.ready = true;
  }
  if (!c->d_flags) {
    int rc;
    if ((rc = upload_raw(c->tab_id, &c->d_tab_id)) || (rc = upload_raw(c->zref, &c->d_zref))) return rc;
    cudaError_t e = cudaMalloc(&c->d_flags, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_min, c->n_sys * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tr, c->n_sys * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (cells)");
  }
  return MBS_OK;
}

}  // namespace

extern "C" {

int mbs_cells_create(const mbs_qm_desc *qms, int n_sys, double dt, long long n_steps, const mbs_source *drives,
                     int record_every, mbs_cells_t *out) {
  g_err.clear();
  if (!out) return fail(MBS_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!qms || !drives || n_sys < 1) return fail(MBS_E_INVALID, "need n_sys >= 1 systems and their drives");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(MBS_E_INVALID, "dt must be > 0");
  if (n_steps < 1 || n_steps > (1LL << 31)) return fail(MBS_E_INVALID, "n_steps must be in [1, 2^31]");
  if (record_every < 1) return fail(MBS_E_INVALID, "record_every must be >= 1");
  const int N = qms[0].n_levels;
  if (N != 2 && N != 3) return fail(MBS_E_INVALID, "driven cells: n_levels must be 2 or 3");
  auto c = std::make_unique<mbs_cells_s>();
  c->N = N;
  c->K = N * N - 1;
  c->P = N * (N - 1) / 2;
  c->n_sys = n_sys;
  c->dt = dt;
  c->nt = n_steps;
  c->every = record_every;
  c->n_rec = n_steps / record_every;
  const int K = c->K, P = c->P, N2 = N * N;
  c->rows = K * K + K + 3 * P + N * (K + 1);
  c->prm.assign((size_t)c->rows * n_sys, 0.0);
  c->zref.assign((size_t)n_sys * N2, 0.0);
  c->Dinit.assign((size_t)K * n_sys, 0.0);
  c->amp.assign(n_sys, 0.0);
  c->tab_id.assign(n_sys, 0);
  int status = MBS_OK;
  // drive shapes: systems with the same (tau, t0, omega, phase) share one
  std::vector<std::array<double, 5>> shapes;
  for (int s = 0; s < n_sys; ++s) {
    const mbs_source &d = drives[s];
    if (!std::isfinite(d.e0) || !std::isfinite(d.tau) || !std::isfinite(d.t0) || !std::isfinite(d.omega) ||
        !std::isfinite(d.phase) || !(d.tau > 0))
      return fail(MBS_E_INVALID, "system %d: drive parameters must be finite with tau > 0", s);
    if (d.shape != MBS_SHAPE_SECH && d.shape != MBS_SHAPE_GAUSS) return fail(MBS_E_INVALID, "system %d: bad shape", s);
    const std::array<double, 5> k{d.tau, d.t0, d.omega, d.phase, (double)d.shape};
    int id = -1;
    for (size_t j = 0; j < shapes.size() && id < 0; ++j)
      if (shapes[j] == k) id = (int)j;
    if (id < 0) {
      id = (int)shapes.size();
      shapes.push_back(k);
    }
    c->tab_id[s] = id;
    c->amp[s] = d.e0;
  }
  c->n_tab = (int)shapes.size();
  // E^n = e0 envelope((t_n - t0)/tau) sin(omega t_n + phase), t_n = n dt; E^0 = 0
  c->tab.assign((size_t)c->n_tab * n_steps, 0.0);
  for (int j = 0; j < c->n_tab; ++j)
    for (long long n = 1; n < n_steps; ++n) {
      const double t = (double)n * dt;
      c->tab[(size_t)j * n_steps + n] =
          std::sin(shapes[j][2] * t + shapes[j][3]) * envelope((int)shapes[j][4], (t - shapes[j][1]) / shapes[j][0]);
    }
  std::vector<int> codes(n_sys, MBS_OK);
  std::vector<std::string> msgs(n_sys);
#pragma omp parallel for schedule(dynamic, 16)
  for (int s = 0; s < n_sys; ++s) {
    if (qms[s].n_levels != N) {
      codes[s] = MBS_E_INVALID;
      msgs[s] = "all systems must have the same number of levels";
      continue;
    }
    QDesc q;
    const int rc = build_qdesc(qms[s], q);
    if (rc < 0) {
      codes[s] = rc;
      msgs[s] = g_err;
      continue;
    }
    codes[s] = rc;
    Step st;
    build_step(q, 1.0, dt, st);
    auto put = [&](int row, double v) { c->prm[(size_t)row * n_sys + s] = v; };
    for (int i = 0; i < K * K; ++i) put(i, st.AKm1[i]);
    for (int i = 0; i < K; ++i) put(K * K + i, st.c[i]);
    int p = 0;
    for (int j = 0; j < N; ++j)
      for (int k = j + 1; k < N; ++k, ++p) {
        put(K * K + K + p, (q.lambda[j] - q.lambda[k]) * dt / kHbar);
        put(K * K + K + P + 2 * p, q.yref[N + 2 * p]);
        put(K * K + K + P + 2 * p + 1, q.yref[N + 2 * p + 1]);
      }
    for (int k = 0; k < N; ++k) {   // rho_kk^{n+1/2} = coef . u + coef_K
      const std::vector<double> h = rho_functional(q, k, k, false);
      std::vector<double> hA(N2, 0.0);
      for (int cc = 0; cc < N2; ++cc)
        for (int r = 0; r < N2; ++r) hA[cc] += h[r] * st.Ah[r * N2 + cc];
      double h0 = 0;
      for (int cc = 0; cc < N2; ++cc) h0 += hA[cc] * q.yref[cc];
      const int r0 = K * K + K + 3 * P + k * (K + 1);
      for (int i = 0; i < K; ++i) put(r0 + i, hA[full_of(N, i)] - (i < N - 1 ? hA[N - 1] : 0.0));
      put(r0 + K, h0);
    }
    std::vector<double> x0(N2, 0.0);
    for (int i = 0; i < N2; ++i)
      for (int j = 0; j < N2; ++j) x0[i] += st.Ehm1[i * N2 + j] * q.yinit[j];
    for (int i = 0; i < K; ++i)
      c->Dinit[(size_t)i * n_sys + s] = x0[full_of(N, i)] + (q.yinit[full_of(N, i)] - q.yref[full_of(N, i)]);
    std::copy(q.yref.begin(), q.yref.end(), &c->zref[(size_t)s * N2]);
  }
  for (int s = 0; s < n_sys; ++s) {
    if (codes[s] < 0) return fail(codes[s], "system %d: %s", s, msgs[s].c_str());
    if (codes[s] == MBS_W_NOT_PSD) status = MBS_W_NOT_PSD;
  }
  for (double v : c->prm)
    if (!std::isfinite(v)) return fail(MBS_E_NUMERIC, "non-finite step operator (check H0, mu, rates and dt)");
  *out = c.release();
  return status;
}

int mbs_cells_solve(mbs_cells_t c, int precision, void *cuda_stream) {
  g_err.clear();
  if (!c) return fail(MBS_E_INVALID, "cells is NULL");
  if (precision != MBS_PREC_FP64 && precision != MBS_PREC_FP32) return fail(MBS_E_INVALID, "bad precision");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int rc = cells_device(c, precision);
  if (rc) return rc;
  auto &b = c->b[precision];
  const size_t rb = rsize(precision), ns = (size_t)c->n_sys;
  cudaError_t e;
  if (precision == 0) {
    e = cudaMemcpyAsync(b.D, c->Dinit.data(), c->Dinit.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  } else {
    std::vector<float> f(c->Dinit.begin(), c->Dinit.end());
    e = cudaMemcpyAsync(b.D, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // f leaves scope
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b.C, 0, ns * c->K * rb, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_flags, 0, 4 * sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "cells state reset");
  mbs::CellsArgs a{};
  a.prec = precision;
  a.N = c->N;
  a.n_sys = c->n_sys;
  a.nt = c->nt;
  a.every = c->every;
  a.prm = b.prm;
  a.D = b.D;
  a.C = b.C;
  a.amp = b.amp;
  a.tab_id = c->d_tab_id;
  a.tab = b.tab;
  a.tab_stride = precision == 0 ? c->nt : 2 * c->nt;
  a.rec = b.rec;
  a.zref = c->d_zref;
  a.flags = c->d_flags;
  constexpr long long CHUNK = 2048;   // steps per launch
  for (long long n0 = 0; n0 < c->nt; n0 += CHUNK) {
    const int ns_ = (int)std::min<long long>(CHUNK, c->nt - n0);
    if ((rc = mbs::launch_cells(a, n0, ns_, st))) return cuda_fail((cudaError_t)rc, "cells launch");
  }
  if ((rc = mbs::launch_cells_check(a, c->d_min, c->d_tr, st))) return cuda_fail((cudaError_t)rc, "cells check");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cells solve");
  int flags[4];
  std::vector<double> mn(c->n_sys), tr(c->n_sys);
  if ((e = cudaMemcpy(flags, c->d_flags, sizeof flags, cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(mn.data(), c->d_min, ns * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(tr.data(), c->d_tr, ns * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cells check results");
  c->solved_prec = precision;
  c->st_min = *std::min_element(mn.begin(), mn.end());
  c->st_trace = *std::max_element(tr.begin(), tr.end());
  if (flags[0]) return fail(MBS_E_NUMERIC, "non-finite density matrix");
  if (c->st_min < -1e-6) return fail(MBS_E_NUMERIC, "density matrix eigenvalue %.3g < -1e-6", c->st_min);
  return MBS_OK;
}

int mbs_cells_fetch(mbs_cells_t c, int sys, double *out, size_t cap, size_t *n_written) {
  g_err.clear();
  if (!c) return fail(MBS_E_INVALID, "cells is NULL");
  if (sys < 0 || sys >= c->n_sys) return fail(MBS_E_INVALID, "system index out of range");
  const size_t n = (size_t)c->n_rec * c->N;
  if (n_written) *n_written = n;
  if (!out) return MBS_OK;
  if (cap < n) return fail(MBS_E_INVALID, "capacity %zu < %zu", cap, n);
  if (c->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  if (n == 0) return MBS_OK;
  const size_t rb = rsize(c->solved_prec);
  // element (r, k) of system sys sits at (r N + k) n_sys + sys
  const char *src = static_cast<const char *>(c->b[c->solved_prec].rec) + (size_t)sys * rb;
  cudaError_t e;
  if (c->solved_prec == 0) {
    e = cudaMemcpy2D(out, rb, src, (size_t)c->n_sys * rb, rb, n, cudaMemcpyDeviceToHost);
  } else {
    std::vector<float> f(n);
    e = cudaMemcpy2D(f.data(), rb, src, (size_t)c->n_sys * rb, rb, n, cudaMemcpyDeviceToHost);
    for (size_t i = 0; i < n; ++i) out[i] = f[i];
  }
  if (e != cudaSuccess) return cuda_fail(e, "cells fetch");
  return MBS_OK;
}

int mbs_cells_stats(mbs_cells_t c, double *max_trace_dev, double *min_eig) {
  g_err.clear();
  if (!c) return fail(MBS_E_INVALID, "cells is NULL");
  if (c->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  if (max_trace_dev) *max_trace_dev = c->st_trace;
  if (min_eig) *min_eig = c->st_min;
  return MBS_OK;
}

void mbs_cells_destroy(mbs_cells_t c) {
  if (!c) return;
  free_cells(c);
  delete c;
}

}  // extern "C"
