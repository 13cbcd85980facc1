// mbs_step_math.h -- the FP64 step operators of one cell (Sec. 2.2 operator
// splitting), as plain arithmetic on fixed-size arrays, compiled both for
// the host (mbs_setup.cpp) and for the device (mbs_setup_dev.cu, the
// per-cell operators of jittered two-level media), so that the two setups
// run the same formulas.
//
// The coordinates are those of mbs_internal.h: y = the real coordinates of
// rho~ = V^+ rho V (N populations, then the (Re, Im) of each coherence
// pair); the Liouvillian is M = hfac MH + MD (MH from H0, MD from the
// dissipator), a real N^2 x N^2 matrix.  Deviation coordinates drop the last
// population (it is 1 minus the others): component i of the K = N^2 - 1
// deviation components is full coordinate fo(i) = i < N - 1 ? i : i + 1.
#pragma once

#ifdef __CUDACC__
#define MBS_HD __host__ __device__
#else
#define MBS_HD
#endif

namespace mbs_math {

MBS_HD inline double absd(double x) { return x < 0 ? -x : x; }

// c = a b for n x n row-major matrices (rows of b streamed into c)
template <int n>
MBS_HD inline void rmatmul_n(const double *a, const double *b, double *c) {
  for (int i = 0; i < n; ++i) {
    double r[n];
    for (int j = 0; j < n; ++j) r[j] = 0.0;
    for (int k = 0; k < n; ++k) {
      const double x = a[i * n + k];
      for (int j = 0; j < n; ++j) r[j] += x * b[k * n + j];
    }
    for (int j = 0; j < n; ++j) c[i * n + j] = r[j];
  }
}

// exp(A) - I for a real n x n matrix, accurate relative to itself: scale by
// 2^-s until ||A||_1 <= 1/4, evaluate the Taylor series without its leading
// identity in nested (Horner) form,
//   exp(B) - I = B (I + B/2 (I + B/3 (... (I + B/m)))),
// with the smallest m whose truncation bound ||B||^m / (m + 1)! stays below
// 2^-70 (at most 16 terms at ||B|| = 1/4), and undo the scaling with the
// squarings in the same form, exp(2B) - I = E (E + 2 I) for E = exp(B) - I.
// The step operators act on small deviations through exp(L0 dt) - I, whose
// entries are ~|L0| dt; forming exp(L0 dt) first and subtracting I would
// leave them with an absolute error of one ulp of 1 -- a systematic error
// repeated every step.  A non-finite A gives NaN everywhere.
template <int n>
MBS_HD inline void expm1_horner(const double *A, double *E) {
  double nrm = 0;
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int i = 0; i < n; ++i) s += absd(A[i * n + j]);
    nrm = s > nrm ? s : nrm;
  }
  if (!(nrm - nrm == 0.0)) {   // inf or NaN
    for (int i = 0; i < n * n; ++i) E[i] = nrm - nrm;
    return;
  }
  int sq = 0;
  double sc = 1.0;   // 2^-sq, exact
  while (nrm > 0.25) {
    nrm *= 0.5;
    sc *= 0.5;
    ++sq;
  }
  int m = 1;
  for (double bound = nrm / 2.0; m < 20 && bound > 0x1p-70; bound *= nrm / (m + 2)) ++m;
  double B[n * n], P[n * n], T[n * n];
  for (int i = 0; i < n * n; ++i) {
    B[i] = A[i] * sc;
    P[i] = B[i] / m;
  }
  for (int k = m - 1; k >= 1; --k) {
    for (int i = 0; i < n; ++i) P[i * n + i] += 1.0;
    rmatmul_n<n>(B, P, T);
    const double rk = 1.0 / k;   // one division per term (each product rounds once more)
    for (int i = 0; i < n * n; ++i) P[i] = T[i] * rk;
  }
  for (int k = 0; k < sq; ++k) {
    rmatmul_n<n>(P, P, T);
    for (int i = 0; i < n * n; ++i) P[i] = T[i] + 2.0 * P[i];
  }
  for (int i = 0; i < n * n; ++i) E[i] = P[i];
}

// One step's operators for N levels (K = N^2 - 1 deviation components):
//   Ehm1 = exp(L0 dt/2) - I and Ah = exp(L0 dt/2) on the full coordinates;
//   AKm1 = exp(L0 dt) - I on the deviations (formed as Eh (Eh + 2 I));
//   c = (exp(L0 dt) - I) yref, the affine offset at the reference state;
//   g, g0: d_t P / n3D = tr(mu L0 exp(L0 dt/2) v) = sum_j lambda_j [M Ah y]_j
//   as a functional of the deviation (g) plus its constant part (g0).
template <int N>
struct StepOps {
  static constexpr int N2 = N * N, K = N2 - 1;
  double AKm1[K * K], c[K], g[K], g0, Ah[N2 * N2], Ehm1[N2 * N2];
};

template <int N>
MBS_HD inline void step_ops(const double *MH, const double *MD, const double *yref, const double *lambda, double hfac,
                            double dt, StepOps<N> &o) {
  constexpr int N2 = N * N, K = N2 - 1;
  double M[N2 * N2], Mh[N2 * N2], Em1[N2 * N2], MAh[N2 * N2], ay[N2], gf[N2];
  for (int i = 0; i < N2 * N2; ++i) {
    M[i] = hfac * MH[i] + MD[i];
    Mh[i] = 0.5 * dt * M[i];
  }
  expm1_horner<N2>(Mh, o.Ehm1);
  rmatmul_n<N2>(o.Ehm1, o.Ehm1, Em1);
  for (int i = 0; i < N2 * N2; ++i) {
    Em1[i] += 2.0 * o.Ehm1[i];
    o.Ah[i] = o.Ehm1[i];
  }
  for (int i = 0; i < N2; ++i) o.Ah[i * N2 + i] += 1.0;
  for (int i = 0; i < K; ++i) {
    const int fi = i < N - 1 ? i : i + 1;
    for (int j = 0; j < K; ++j) {
      const int fj = j < N - 1 ? j : j + 1;
      o.AKm1[i * K + j] = Em1[fi * N2 + fj] - (j < N - 1 ? Em1[fi * N2 + N - 1] : 0.0);
    }
  }
  for (int i = 0; i < N2; ++i) {
    ay[i] = 0.0;
    for (int j = 0; j < N2; ++j) ay[i] += Em1[i * N2 + j] * yref[j];
  }
  for (int i = 0; i < K; ++i) o.c[i] = ay[i < N - 1 ? i : i + 1];
  rmatmul_n<N2>(M, o.Ah, MAh);
  for (int c = 0; c < N2; ++c) gf[c] = 0.0;
  for (int j = 0; j < N; ++j)
    for (int c = 0; c < N2; ++c) gf[c] += lambda[j] * MAh[j * N2 + c];
  for (int i = 0; i < K; ++i) o.g[i] = gf[i < N - 1 ? i : i + 1] - (i < N - 1 ? gf[N - 1] : 0.0);
  o.g0 = 0;
  for (int c = 0; c < N2; ++c) o.g0 += gf[c] * yref[c];
}

// The structured two-level rows of one cell from its dense rows (A - I, the
// offset c, the coupling w, w0): true and the 7 rows a00, a02, a11, a20,
// a22, w0, w2 when A - I has the optical-Bloch pattern (non-zero only at
// (0,0), (0,2), (1,1), (2,0), (2,2)), the offset vanishes and the coupling
// has no (1) component and no constant (relative thresholds 1e-13).
MBS_HD inline bool bloch2_rows(const double *A, const double *c, const double *w, double w0, double *rows) {
  double amax = 0, wmax = 0;
  for (int r = 0; r < 9; ++r) amax = absd(A[r]) > amax ? absd(A[r]) : amax;
  for (int r = 0; r < 3; ++r) wmax = absd(w[r]) > wmax ? absd(w[r]) : wmax;
  const double ta = 1e-13 * amax, tw = 1e-13 * wmax;
  if (absd(A[1]) > ta || absd(A[3]) > ta || absd(A[5]) > ta || absd(A[7]) > ta || absd(c[0]) > 1e-13 ||
      absd(c[1]) > 1e-13 || absd(c[2]) > 1e-13 || absd(w[1]) > tw || absd(w0) > tw)
    return false;
  rows[0] = A[0];
  rows[1] = A[2];
  rows[2] = A[4];
  rows[3] = A[6];
  rows[4] = A[8];
  rows[5] = w[0];
  rows[6] = w[2];
  return true;
}

}  // namespace mbs_math
