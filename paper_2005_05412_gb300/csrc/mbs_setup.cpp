// mbs_setup.cpp -- FP64 host setup of the per-material step operators
// (Sec. 2.2 operator splitting, Sec. 3.1.1 Lindblad relaxation):
//   * mu = V diag(lambda) V^+ by Householder reduction of the Hermitian
//     matrix to real symmetric tridiagonal form followed by implicit QL
//     iterations (Golub & Van Loan, Secs. 8.3 and 8.5);
//   * the Liouvillian L0 (H0 and the dissipator of Eq. lindbladdiss) as a
//     real matrix on the coordinates of rho~ = V^+ rho V (mbs_internal.h);
//     the rate form (Eq. relax_pop, pure dephasing) becomes Lindblad
//     operators |i><j| and diag(v_k), the latter from the double-centred
//     dephasing matrix G = -1/2 J D J (D_ij = 2 gamma_ij,p), which is PSD iff
//     the dephasing rates admit a PSD coefficient matrix;
//   * exp(L0 dt) - I and exp(L0 dt/2) - I by Taylor series without the
//     identity, with scaling and squaring in the same form;
//   * the steady state of L0 (when unique) as the deviation reference.
#include <algorithm>
#include <array>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "mbs_host_internal.h"
#include "mbs_step_math.h"

namespace mbs_host {

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

// exp(A) - I for the Liouville-space sizes N^2 (N = 2..6): mbs_math::expm1_horner
// (mbs_step_math.h: scaling, nested Taylor series without the identity,
// squarings in the same form)
void expm1_taylor(int n, const double *A, double *E) {
  switch (n) {
    case 4: return mbs_math::expm1_horner<4>(A, E);
    case 9: return mbs_math::expm1_horner<9>(A, E);
    case 16: return mbs_math::expm1_horner<16>(A, E);
    case 25: return mbs_math::expm1_horner<25>(A, E);
    case 36: return mbs_math::expm1_horner<36>(A, E);
    default: break;
  }
  for (int i = 0; i < n * n; ++i) E[i] = std::nan("");   // not a Liouville-space size
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


// One step's FP64 operators for a level count known at compile time
// (mbs_math::step_ops, the arithmetic the device setup of jittered two-level
// media runs too); the Step's vectors keep their capacity when the caller
// reuses it (one call per cell for jittered media).
template <int N>
static void build_step_n(const QDesc &q, double hfac, double dt, Step &s) {
  constexpr int N2 = N * N, K = N2 - 1;
  mbs_math::StepOps<N> o;
  mbs_math::step_ops<N>(q.MH.data(), q.MD.data(), q.yref.data(), q.lambda.data(), hfac, dt, o);
  s.Ah.assign(o.Ah, o.Ah + N2 * N2);
  s.Ehm1.assign(o.Ehm1, o.Ehm1 + N2 * N2);
  s.AKm1.assign(o.AKm1, o.AKm1 + K * K);
  s.AK.assign(o.AKm1, o.AKm1 + K * K);
  for (int i = 0; i < K; ++i) s.AK[i * K + i] += 1.0;
  s.c.assign(o.c, o.c + K);
  s.g.assign(o.g, o.g + K);
  s.g0 = o.g0;
}

void build_step(const QDesc &q, double hfac, double dt, Step &s) {
  switch (q.N) {
    case 2: return build_step_n<2>(q, hfac, dt, s);
    case 3: return build_step_n<3>(q, hfac, dt, s);
    case 4: return build_step_n<4>(q, hfac, dt, s);
    case 5: return build_step_n<5>(q, hfac, dt, s);
    case 6: return build_step_n<6>(q, hfac, dt, s);
    default: break;
  }
  s = Step();   // no level count outside 2..6 reaches here (build_qdesc rejects it)
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

}  // namespace mbs_host
