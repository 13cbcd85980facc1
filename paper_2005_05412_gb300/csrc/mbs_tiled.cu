// mbs_tiled.cu -- temporally tiled kernels (N = 2, 3) and their launcher.
#include "mbs_device.cuh"

namespace mbs {
using namespace dev;

int tiled_supported(int prec, int N) { return (N == 2 || N == 3) && (prec == 0 || prec == 1); }

int launch_tiled(const Args &a, long long n0, int nsteps, int T, int cur, void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const bool pc = a.pcell != nullptr, b2 = a.pcell2 != nullptr;
  if (a.N == 2) {
    if (a.prec == 0) {
      if (b2) return tiled_impl<double, 2, 4, false, 2>(a, n0, nsteps, T, cur, st);
      return pc ? tiled_impl<double, 2, 4, false, 1>(a, n0, nsteps, T, cur, st)
                : tiled_impl<double, 2, 4, false, 0>(a, n0, nsteps, T, cur, st);
    }
    if (b2) return tiled_impl<float, 2, 4, true, 2>(a, n0, nsteps, T, cur, st);
    return pc ? tiled_impl<float, 2, 4, true, 1>(a, n0, nsteps, T, cur, st)
              : tiled_impl<float, 2, 4, true, 0>(a, n0, nsteps, T, cur, st);
  }
  if (a.N == 3 && !pc) {
    if (a.prec == 0) return tiled_impl<double, 3, 2, false, 0>(a, n0, nsteps, T, cur, st);
    return tiled_impl<float, 3, 2, true, 0>(a, n0, nsteps, T, cur, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace mbs
