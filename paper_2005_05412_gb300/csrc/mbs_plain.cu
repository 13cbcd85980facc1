// mbs_plain.cu -- plain (Algorithm 1) step and state check for N in {2, 3}.
#include "mbs_device.cuh"

namespace mbs {
using namespace dev;

int plain_step_n23(int N, const Args &a, long long n, int cur, cudaStream_t st) {
  switch (N) {
    case 2:
      return a.prec == 0 ? plain_step_impl<double, 2, false>(a, n, cur, st) : plain_step_impl<float, 2, true>(a, n, cur, st);
    case 3:
      return a.prec == 0 ? plain_step_impl<double, 3, false>(a, n, cur, st) : plain_step_impl<float, 3, true>(a, n, cur, st);
  }
  return (int)cudaErrorInvalidValue;
}

int check_n23(int N, const Args &a, int cur, const int *cells, int n_cells, double *mn, double *tr,
              const double *z, cudaStream_t st) {
  switch (N) {
    case 2:
      return a.prec == 0 ? check_impl<double, 2>(a, cur, cells, n_cells, mn, tr, z, st) : check_impl<float, 2>(a, cur, cells, n_cells, mn, tr, z, st);
    case 3:
      return a.prec == 0 ? check_impl<double, 3>(a, cur, cells, n_cells, mn, tr, z, st) : check_impl<float, 3>(a, cur, cells, n_cells, mn, tr, z, st);
  }
  return (int)cudaErrorInvalidValue;
}

int plain_step_n45(int N, const Args &a, long long n, int cur, cudaStream_t st);
int check_n45(int N, const Args &a, int cur, const int *cells, int n_cells, double *mn, double *tr, const double *z,
              cudaStream_t st);
int plain_step_n6(int N, const Args &a, long long n, int cur, cudaStream_t st);
int sweep_n45(int N, const Args &a, int dcur, int ecur, int hcur, double tol, cudaStream_t st);
int sweep_n6(int N, const Args &a, int dcur, int ecur, int hcur, double tol, cudaStream_t st);
int check_n6(int N, const Args &a, int cur, const int *cells, int n_cells, double *mn, double *tr, const double *z,
             cudaStream_t st);

int launch_plain_step(const Args &a, long long n, int cur, void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (a.N <= 3) return plain_step_n23(a.N, a, n, cur, st);
  if (a.N <= 5) return plain_step_n45(a.N, a, n, cur, st);
  return plain_step_n6(a.N, a, n, cur, st);
}

int launch_check(const Args &a, int cur, const int *cells, int n_cells, double *out_min_eig, double *out_trace_dev,
                 const void *zref_full, const void *, void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const double *z = reinterpret_cast<const double *>(zref_full);
  if (a.N <= 3) return check_n23(a.N, a, cur, cells, n_cells, out_min_eig, out_trace_dev, z, st);
  if (a.N <= 5) return check_n45(a.N, a, cur, cells, n_cells, out_min_eig, out_trace_dev, z, st);
  return check_n6(a.N, a, cur, cells, n_cells, out_min_eig, out_trace_dev, z, st);
}

int sweep_n23(int N, const Args &a, int dcur, int ecur, int hcur, double tol, cudaStream_t st) {
  switch (N) {
    case 2:
      return a.prec == 0 ? sweep_impl<double, 2>(a, dcur, ecur, hcur, tol, st) : sweep_impl<float, 2>(a, dcur, ecur, hcur, tol, st);
    case 3:
      return a.prec == 0 ? sweep_impl<double, 3>(a, dcur, ecur, hcur, tol, st) : sweep_impl<float, 3>(a, dcur, ecur, hcur, tol, st);
  }
  return (int)cudaErrorInvalidValue;
}

int launch_sweep(const Args &a, int dcur, int ecur, int hcur, double tol, void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (a.N <= 3) return sweep_n23(a.N, a, dcur, ecur, hcur, tol, st);
  if (a.N <= 5) return sweep_n45(a.N, a, dcur, ecur, hcur, tol, st);
  return sweep_n6(a.N, a, dcur, ecur, hcur, tol, st);
}

}  // namespace mbs
