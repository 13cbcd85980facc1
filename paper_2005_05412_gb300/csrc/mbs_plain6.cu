// mbs_plain6.cu -- plain (Algorithm 1) step and state check for N in {6}.
#include "mbs_device.cuh"

namespace mbs {
using namespace dev;

int plain_step_n6(int N, const Args &a, long long n, int cur, cudaStream_t st) {
  switch (N) {
    case 6:
      return a.prec == 0 ? plain_step_impl<double, 6, false>(a, n, cur, st) : plain_step_impl<float, 6, true>(a, n, cur, st);
  }
  return (int)cudaErrorInvalidValue;
}

int check_n6(int N, const Args &a, int cur, const int *cells, int n_cells, double *mn, double *tr,
              const double *z, cudaStream_t st) {
  switch (N) {
    case 6:
      return a.prec == 0 ? check_impl<double, 6>(a, cur, cells, n_cells, mn, tr, z, st) : check_impl<float, 6>(a, cur, cells, n_cells, mn, tr, z, st);
  }
  return (int)cudaErrorInvalidValue;
}

int sweep_n6(int N, const Args &a, int dcur, int ecur, int hcur, double tol, cudaStream_t st) {
  switch (N) {
    case 6:
      return a.prec == 0 ? sweep_impl<double, 6>(a, dcur, ecur, hcur, tol, st) : sweep_impl<float, 6>(a, dcur, ecur, hcur, tol, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace mbs
