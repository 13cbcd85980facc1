// mbs_static.cu -- density-matrix check that allocates no device memory.
//
// Variant of the state-check kernel (k_check): instead of per-cell results
// in scenario-owned scratch buffers reduced on the host, the per-matrix
// results live in a fixed file-scope __device__ array and are reduced on
// the device into the caller's output.  It serves callers that cannot call
// cudaMalloc: a framework that owns every device allocation through its own
// pool, or a loop that must not stall on the device-wide synchronisation an
// allocation can imply.
//
// Every GPU that loads this library holds the scratch array until the
// process exits: 3 doubles per matrix for MBS_STATIC_CHECK_MAX matrices
// (1.5 MB).  Its device address is looked up once per device, on the first
// call with that device current, and cached for the life of the process; a
// cudaDeviceReset invalidates the cached address (do not call the entry point
// on a device after resetting it).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mbs.h"
#include "mbs_device.cuh"

namespace {

// per matrix: smallest eigenvalue, |tr - 1|, non-finite flag
static __device__ __align__(256) double g_check_scratch[3 * MBS_STATIC_CHECK_MAX];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch[kMaxDevices] = {};   // device address of g_check_scratch, per device

template <int N>
__global__ void k_rho_check(const double *rho, int n, double *scratch) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double *r = rho + (size_t)i * 2 * N * N;
  double re[N][N], im[N][N];
  bool finite = true;
  double tr = 0.0;
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      // Hermitian part (rho + rho^+) / 2
      re[a][b] = 0.5 * (r[2 * (a * N + b)] + r[2 * (b * N + a)]);
      im[a][b] = 0.5 * (r[2 * (a * N + b) + 1] - r[2 * (b * N + a) + 1]);
      finite &= isfinite(r[2 * (a * N + b)]) && isfinite(r[2 * (a * N + b) + 1]);
    }
  for (int a = 0; a < N; ++a) tr += r[2 * (a * N + a)];
  double mn = finite ? mbs::dev::min_eig_bisect<N>(re, im) : 0.0;
  finite = finite && isfinite(mn);
  scratch[3 * i] = finite ? mn : 0.0;
  scratch[3 * i + 1] = finite ? fabs(tr - 1.0) : 0.0;
  scratch[3 * i + 2] = finite ? 0.0 : 1.0;
}

// one block: out[0] = min eigenvalue, out[1] = max |tr - 1| (both over the
// finite matrices; out[0] = NaN when there is none), out[2] = number of
// matrices with non-finite entries.  Reads only entries [0, n) of the
// scratch array, which this call's first kernel has just written.
__global__ void k_rho_reduce(const double *scratch, int n, double *out) {
  __shared__ double s_min[256], s_tr[256], s_bad[256];
  double mn = 1e300, tr = 0.0, bad = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    if (scratch[3 * i + 2] == 0.0) mn = fmin(mn, scratch[3 * i]);
    tr = fmax(tr, scratch[3 * i + 1]);
    bad += scratch[3 * i + 2];
  }
  s_min[threadIdx.x] = mn;
  s_tr[threadIdx.x] = tr;
  s_bad[threadIdx.x] = bad;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + w]);
      s_tr[threadIdx.x] = fmax(s_tr[threadIdx.x], s_tr[threadIdx.x + w]);
      s_bad[threadIdx.x] += s_bad[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s_bad[0] < (double)n ? s_min[0] : nan("");
    out[1] = s_tr[0];
    out[2] = s_bad[0];
  }
}

// Device address of the scratch array for the current device, looked up
// once per device (with that device current).
int scratch_for_current_device(double **p) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return mbs::set_error(MBS_E_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return mbs::set_error(MBS_E_INVALID, "device ordinal too large");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    void *addr = nullptr;
    e = cudaGetSymbolAddress(&addr, g_check_scratch);
    if (e != cudaSuccess) return mbs::set_error(MBS_E_CUDA, cudaGetErrorString(e));
    g_scratch[dev] = static_cast<double *>(addr);
  }
  *p = g_scratch[dev];
  return MBS_OK;
}

}  // namespace

extern "C" int mbs_check_rho_static(const double *rho, int n, int n_levels, double *out, void *cuda_stream) {
  if (!rho || !out) return mbs::set_error(MBS_E_INVALID, "rho and out must be device pointers");
  if (n < 1 || n > MBS_STATIC_CHECK_MAX)
    return mbs::set_error(MBS_E_INVALID, "n must be in [1, MBS_STATIC_CHECK_MAX]");
  if (n_levels < 2 || n_levels > mbs::NMAX) return mbs::set_error(MBS_E_INVALID, "n_levels must be in [2, 6]");
  double *scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int bs = 128, gs = (n + bs - 1) / bs;
  switch (n_levels) {
    case 2: k_rho_check<2><<<gs, bs, 0, st>>>(rho, n, scratch); break;
    case 3: k_rho_check<3><<<gs, bs, 0, st>>>(rho, n, scratch); break;
    case 4: k_rho_check<4><<<gs, bs, 0, st>>>(rho, n, scratch); break;
    case 5: k_rho_check<5><<<gs, bs, 0, st>>>(rho, n, scratch); break;
    default: k_rho_check<6><<<gs, bs, 0, st>>>(rho, n, scratch); break;
  }
  k_rho_reduce<<<1, 256, 0, st>>>(scratch, n, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mbs::set_error(MBS_E_CUDA, cudaGetErrorString(e));
  return MBS_OK;
}
