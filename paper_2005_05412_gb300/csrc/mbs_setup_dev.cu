// mbs_setup_dev.cu -- the per-cell FP64 step operators of jittered two-level
// media, formed on the device.  A jittered medium (Sec. 4's SIT example with
// a per-cell transition frequency and density) needs exp(L0 dt/2) - I and
// its derived rows for every cell; on 10^6 cells that is ~30 ms of host
// time against ~1 ms here.  The arithmetic is mbs_math::step_ops, the same
// code the host setup runs (mbs_step_math.h), in FP64; the host forms the
// per-medium parts (the Liouvillian's H0 and dissipator parts MH, MD, the
// dipole eigenvalues, the reference and initial states) as before.
#include <cstdint>

#include "mbs_setup_dev.h"
#include "mbs_step_math.h"

namespace mbs {
namespace {

// one cell per thread; rows as in the host setup: pcell [16][ld] (A - I,
// the offset c, the coupling w = cpl g, w0 = cpl g0), pcell2 [7][ld] (the
// structured rows), dinit [3][ld]; counts[0] = cells with a non-finite
// operator, counts[1] = cells without the optical-Bloch pattern
__global__ void k_setup_cells2(const SetupSlot2 *__restrict__ slots, const uint8_t *__restrict__ mat,
                               const int *__restrict__ qslot, const double *__restrict__ jitter, int nx, int off,
                               int ld, double dt, double *__restrict__ pcell, double *__restrict__ pcell2,
                               double *__restrict__ dinit, int *__restrict__ counts) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nx) return;
  const int sl = qslot[mat[off + m]];
  if (sl < 0) return;   // vacuum: the rows stay zero
  const SetupSlot2 &q = slots[sl];
  constexpr int K = 3;
  mbs_math::StepOps<2> o;
  mbs_math::step_ops<2>(q.MH, q.MD, q.yref, q.lambda, jitter[2 * m + 1], dt, o);
  const double cpl = q.cpl0 * jitter[2 * m];
  const size_t col = (size_t)off + m;
  double w[K];
  for (int i = 0; i < K * K; ++i) pcell[(size_t)i * ld + col] = o.AKm1[i];
  for (int i = 0; i < K; ++i) {
    w[i] = cpl * o.g[i];
    pcell[(size_t)(K * K + i) * ld + col] = o.c[i];
    pcell[(size_t)(K * K + K + i) * ld + col] = w[i];
  }
  const double w0 = cpl * o.g0;
  pcell[(size_t)(K * K + 2 * K) * ld + col] = w0;
  // initial deviation x^0 - yref = (exp(L0 dt/2) - I) yinit + (yinit - yref)
  for (int i = 0; i < K; ++i) {
    const int fi = i < 1 ? i : i + 1;
    double x0 = 0.0;
    for (int j = 0; j < 4; ++j) x0 += o.Ehm1[fi * 4 + j] * q.yinit[j];
    dinit[(size_t)i * ld + col] = x0 + (q.yinit[fi] - q.yref[fi]);
  }
  double rows[7];
  if (mbs_math::bloch2_rows(o.AKm1, o.c, w, w0, rows)) {
    for (int r = 0; r < 7; ++r) pcell2[(size_t)r * ld + col] = rows[r];
  } else {
    atomicAdd(counts + 1, 1);
  }
  const double ak0 = o.AKm1[0] + 1.0;
  if (!(ak0 - ak0 == 0.0)) atomicAdd(counts, 1);
}

__global__ void k_to_float(const double *__restrict__ x, float *__restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

}  // namespace

int setup_cells2(const SetupSlot2 *slots, const uint8_t *mat, const int *qslot, const double *jitter, int nx, int off,
                 int ld, double dt, double *pcell, double *pcell2, double *dinit, int *counts, void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int bs = 128;
  k_setup_cells2<<<(nx + bs - 1) / bs, bs, 0, st>>>(slots, mat, qslot, jitter, nx, off, ld, dt, pcell, pcell2, dinit,
                                                    counts);
  return (int)cudaGetLastError();
}

int to_float(const double *x, float *y, size_t n, void *stream) {
  if (n == 0) return 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int bs = 256;
  const size_t want = (n + bs - 1) / bs;
  const int grid = (int)(want < 152 * 16 ? want : 152 * 16);
  k_to_float<<<grid, bs, 0, st>>>(x, y, n);
  return (int)cudaGetLastError();
}

}  // namespace mbs
