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
      if (b2) return tiled_impl<double, 2, TileGeom<2>::R, false, 2>(a, n0, nsteps, T, cur, st);
      return pc ? tiled_impl<double, 2, TileGeom<2>::R, false, 1>(a, n0, nsteps, T, cur, st)
                : tiled_impl<double, 2, TileGeom<2>::R, false, 0>(a, n0, nsteps, T, cur, st);
    }
    if (b2) return tiled_impl<float, 2, TileGeom<2>::R, true, 2>(a, n0, nsteps, T, cur, st);
    return pc ? tiled_impl<float, 2, TileGeom<2>::R, true, 1>(a, n0, nsteps, T, cur, st)
              : tiled_impl<float, 2, TileGeom<2>::R, true, 0>(a, n0, nsteps, T, cur, st);
  }
  if (a.N == 3 && !pc) {
    if (a.prec == 0) return tiled_impl<double, 3, TileGeom<3>::R, false, 0>(a, n0, nsteps, T, cur, st);
    return tiled_impl<float, 3, TileGeom<3>::R, true, 0>(a, n0, nsteps, T, cur, st);
  }
  return (int)cudaErrorInvalidValue;
}

// Kernel variant of a scenario for the tiled path: (N, PM) with PM as in
// k_tiled; -1 if the tiled path does not cover it.
int tiled_variant(const Args &a) {
  if (a.N == 2) return a.pcell2 ? 2 : (a.pcell ? 1 : 0);
  if (a.N == 3 && !a.pcell) return 0;
  return -1;
}

size_t tiled_batch_smem(int prec, int N, int max_mat_all, int max_slot, int max_qstride) {
  if (prec == 0)
    return N == 2 ? tiled_smem<double, 2, TileGeom<2>::R>(max_mat_all, max_slot, max_qstride)
                  : tiled_smem<double, 3, TileGeom<3>::R>(max_mat_all, max_slot, max_qstride);
  return N == 2 ? tiled_smem<float, 2, TileGeom<2>::R>(max_mat_all, max_slot, max_qstride)
                : tiled_smem<float, 3, TileGeom<3>::R>(max_mat_all, max_slot, max_qstride);
}

int launch_tiled_batch(int prec, int N, int pm, const Args *args, const int2 *tasks, int n_tasks, size_t smem,
                       long long n0, int T, int cur, void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (N == 2) {
    if (prec == 0) {
      if (pm == 2) return tiled_batch_impl<double, 2, TileGeom<2>::R, false, 2>(args, tasks, n_tasks, smem, n0, T, cur, st);
      if (pm == 1) return tiled_batch_impl<double, 2, TileGeom<2>::R, false, 1>(args, tasks, n_tasks, smem, n0, T, cur, st);
      return tiled_batch_impl<double, 2, TileGeom<2>::R, false, 0>(args, tasks, n_tasks, smem, n0, T, cur, st);
    }
    if (pm == 2) return tiled_batch_impl<float, 2, TileGeom<2>::R, true, 2>(args, tasks, n_tasks, smem, n0, T, cur, st);
    if (pm == 1) return tiled_batch_impl<float, 2, TileGeom<2>::R, true, 1>(args, tasks, n_tasks, smem, n0, T, cur, st);
    return tiled_batch_impl<float, 2, TileGeom<2>::R, true, 0>(args, tasks, n_tasks, smem, n0, T, cur, st);
  }
  if (N == 3 && pm == 0) {
    if (prec == 0) return tiled_batch_impl<double, 3, TileGeom<3>::R, false, 0>(args, tasks, n_tasks, smem, n0, T, cur, st);
    return tiled_batch_impl<float, 3, TileGeom<3>::R, true, 0>(args, tasks, n_tasks, smem, n0, T, cur, st);
  }
  return (int)cudaErrorInvalidValue;
}

int launch_sweep_batch(int prec, int N, const Args *args, const int2 *tasks, int n_tasks, int own, long long n0,
                       int cur, double tol, void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (N == 2)
    return prec == 0 ? sweep_batch_impl<double, 2>(args, tasks, n_tasks, own, n0, cur, tol, st)
                     : sweep_batch_impl<float, 2>(args, tasks, n_tasks, own, n0, cur, tol, st);
  if (N == 3)
    return prec == 0 ? sweep_batch_impl<double, 3>(args, tasks, n_tasks, own, n0, cur, tol, st)
                     : sweep_batch_impl<float, 3>(args, tasks, n_tasks, own, n0, cur, tol, st);
  return (int)cudaErrorInvalidValue;
}

}  // namespace mbs
