// mbs_cells.cu -- batched single-cell Lindblad solver (Nx = 1).
//
// With one grid point the method reduces to the master equation of a quantum
// system driven by a prescribed field (Sec. 2.1: the borderline case
// Nx = 1, a solver for the Lindblad equation; application example of the
// V-type three-level system, Sec. 4).  Each thread advances one independent
// system through its whole time loop with the same Strang step as the grid
// kernels (mbs_device.cuh: rotation by the field in the dipole eigenbasis,
// merged constant propagator on the Bloch deviation, Kahan-compensated in
// FP32).  In FP32 the system's step operator lives in registers; in FP64 it
// is read from its column of the parameter table each step.
#include "mbs_device.cuh"

namespace mbs {
namespace dev {

// all step parameters of one system in registers (the coupling is not
// needed: nothing feeds back into the prescribed field)
template <typename real, int N>
struct PrmSys {
  static constexpr int K = N * N - 1, P = N * (N - 1) / 2;
  real a[K * K], cc[K], kp[P], z[2 * P];
  __device__ __forceinline__ real am1(int i, int j) const { return a[i * K + j]; }
  __device__ __forceinline__ real c(int i) const { return cc[i]; }
  __device__ __forceinline__ real w(int) const { return real(0); }
  __device__ __forceinline__ real w0() const { return real(0); }
  __device__ __forceinline__ real kap(int q) const { return kp[q]; }
  __device__ __forceinline__ real zr(int i) const { return z[i]; }
};

// the same, read from the system's column of the table at every use
template <typename real, int N>
struct PrmSysCol {
  static constexpr int K = N * N - 1, P = N * (N - 1) / 2;
  const real *p;   // &prm[0][sys]
  int ld;          // systems (the table's row length)
  __device__ __forceinline__ real am1(int i, int j) const { return p[(size_t)(i * K + j) * ld]; }
  __device__ __forceinline__ real c(int i) const { return p[(size_t)(K * K + i) * ld]; }
  __device__ __forceinline__ real w(int) const { return real(0); }
  __device__ __forceinline__ real w0() const { return real(0); }
  __device__ __forceinline__ real kap(int q) const { return p[(size_t)(K * K + K + q) * ld]; }
  __device__ __forceinline__ real zr(int i) const { return p[(size_t)(K * K + K + P + i) * ld]; }
};

// Steps n0 .. n0 + nsteps - 1 of every system.  Parameter table rows
// (CellsArgs::prm, [rows][n_sys]): A - I (K*K) | c (K) | kap (P) | zr (2P) |
// population functionals N x (K + 1).  Field of system s at step n:
// amp[s] * tab[tab_id[s]][n] (FP32 tables hold high and low words).
// FP32 (parameters in registers) fits 128 registers without spilling: four
// blocks of 128 threads per SM.
template <typename real, int N, bool KAHAN, bool REG>
__global__ void __launch_bounds__(128, REG ? 4 : 1) k_cells(const CellsArgs a, long long n0, int nsteps) {
  constexpr int K = N * N - 1, P = N * (N - 1) / 2;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n_sys) return;
  const real *prm = reinterpret_cast<const real *>(a.prm) + s;
  real *D = reinterpret_cast<real *>(a.D) + s;
  real *Cc = reinterpret_cast<real *>(a.C) + s;
  real d[K], cc[K], u[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    d[i] = D[(size_t)i * a.n_sys];
    cc[i] = KAHAN ? Cc[(size_t)i * a.n_sys] : real(0);
  }
  PrmSys<real, N> qr;
  if constexpr (REG) {
#pragma unroll
    for (int i = 0; i < K * K; ++i) qr.a[i] = prm[(size_t)i * a.n_sys];
#pragma unroll
    for (int i = 0; i < K; ++i) qr.cc[i] = prm[(size_t)(K * K + i) * a.n_sys];
#pragma unroll
    for (int i = 0; i < P; ++i) qr.kp[i] = prm[(size_t)(K * K + K + i) * a.n_sys];
#pragma unroll
    for (int i = 0; i < 2 * P; ++i) qr.z[i] = prm[(size_t)(K * K + K + P + i) * a.n_sys];
  }
  const PrmSysCol<real, N> qc{prm, a.n_sys};
  const real *pop = prm + (size_t)(K * K + K + 3 * P) * a.n_sys;   // N x (K + 1) rows
  const real amp = reinterpret_cast<const real *>(a.amp)[s];
  const real *tab = reinterpret_cast<const real *>(a.tab) + (size_t)a.tab_id[s] * a.tab_stride;
  real *rec = reinterpret_cast<real *>(a.rec);
  // step n records when (n + 1) % every == 0, into record (n + 1) / every - 1:
  // the phase and quotient of n + 1 are carried from step to step (no
  // 64-bit division in the loop)
  long long q = (n0 + 1) / a.every;
  int ph = (int)((n0 + 1) % a.every);
#pragma unroll 1
  for (int t = 0; t < nsteps; ++t) {
    const long long n = n0 + t;
    real fh, fl;
    src_val<real>(tab, n, a.nt, fh, fl);
    const real e = amp * fld_val<real>(fh, fl);
    if constexpr (REG)
      bloch_step<real, N, KAHAN>(qr, e, d, cc, u);
    else
      bloch_step<real, N, KAHAN>(qc, e, d, cc, u);
    if (ph == 0) {
      const long long r = q - 1;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        real v = pop[(size_t)(k * (K + 1) + K) * a.n_sys];
#pragma unroll
        for (int i = 0; i < K; ++i) v += pop[(size_t)(k * (K + 1) + i) * a.n_sys] * u[i];
        rec[((size_t)r * N + k) * a.n_sys + s] = v;
      }
    }
    if (++ph == a.every) {
      ph = 0;
      ++q;
    }
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    D[(size_t)i * a.n_sys] = d[i];
    if (KAHAN) Cc[(size_t)i * a.n_sys] = cc[i];
  }
}

// Final state check of every system: the density matrix x (true value
// delta - compensation on the reference zref[s]) -> |tr - 1| and the smallest
// eigenvalue (inertia bisection); non-finite values set flags[0].
template <typename real, int N>
__global__ void k_cells_check(const CellsArgs a, double *min_eig, double *tr_dev) {
  constexpr int K = N * N - 1, NP = N - 1;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.n_sys) return;
  const real *D = reinterpret_cast<const real *>(a.D) + s;
  const real *Cc = reinterpret_cast<const real *>(a.C) + s;
  const double *zref = a.zref + (size_t)s * N * N;
  double y[N * N], popsum = 0.0;
  bool finite = true;
  for (int i = 0; i < K; ++i) {
    double v = (double)D[(size_t)i * a.n_sys];
    if (a.prec == 1) v -= (double)Cc[(size_t)i * a.n_sys];
    finite &= isfinite(v);
    const int fi = i < NP ? i : i + 1;
    y[fi] = zref[fi] + v;
    if (i < NP) popsum += v;
  }
  y[NP] = zref[NP] - popsum;
  double re[N][N], im[N][N], tr = 0.0;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) re[i][j] = im[i][j] = 0.0;
  for (int i = 0; i < N; ++i) {
    re[i][i] = y[i];
    tr += y[i];
  }
  int q = 0;
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j, ++q) {
      re[i][j] = re[j][i] = y[N + 2 * q];
      im[i][j] = y[N + 2 * q + 1];
      im[j][i] = -y[N + 2 * q + 1];
    }
  double mn = min_eig_bisect<N>(re, im);
  if (!finite || !isfinite(mn)) {
    atomicOr(a.flags, 1);
    mn = -1e300;
  }
  min_eig[s] = mn;
  tr_dev[s] = fabs(tr - 1.0);
}

template <typename real, int N>
int cells_impl(const CellsArgs &a, long long n0, int nsteps, cudaStream_t st) {
  const int bs = 128, gs = (a.n_sys + bs - 1) / bs;
  if constexpr (sizeof(real) == 4)
    k_cells<real, N, true, true><<<gs, bs, 0, st>>>(a, n0, nsteps);
  else
    k_cells<real, N, false, false><<<gs, bs, 0, st>>>(a, n0, nsteps);
  return (int)cudaGetLastError();
}

template <typename real, int N>
int cells_check_impl(const CellsArgs &a, double *mn, double *tr, cudaStream_t st) {
  const int bs = 128, gs = (a.n_sys + bs - 1) / bs;
  k_cells_check<real, N><<<gs, bs, 0, st>>>(a, mn, tr);
  return (int)cudaGetLastError();
}

}  // namespace dev

int launch_cells(const CellsArgs &a, long long n0, int nsteps, void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (a.N == 2) return a.prec == 0 ? dev::cells_impl<double, 2>(a, n0, nsteps, st) : dev::cells_impl<float, 2>(a, n0, nsteps, st);
  if (a.N == 3) return a.prec == 0 ? dev::cells_impl<double, 3>(a, n0, nsteps, st) : dev::cells_impl<float, 3>(a, n0, nsteps, st);
  return (int)cudaErrorInvalidValue;
}

int launch_cells_check(const CellsArgs &a, double *min_eig, double *tr_dev, void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (a.N == 2)
    return a.prec == 0 ? dev::cells_check_impl<double, 2>(a, min_eig, tr_dev, st)
                       : dev::cells_check_impl<float, 2>(a, min_eig, tr_dev, st);
  if (a.N == 3)
    return a.prec == 0 ? dev::cells_check_impl<double, 3>(a, min_eig, tr_dev, st)
                       : dev::cells_check_impl<float, 3>(a, min_eig, tr_dev, st);
  return (int)cudaErrorInvalidValue;
}

}  // namespace mbs
