// mbs_peaks.cu -- arithmetic peaks of the GPU this library runs on, measured
// by small kernels, as denominators of the rooflines of the hot-path kernels:
//
//   FP32 FMA     k_peak_ffma: 8 independent fmaf chains per thread, 8 warps
//                per block, 8 blocks per SM; the FP32 lanes are also the
//                instruction-issue limit (one warp instruction per scheduler
//                and clock), so this rate / 64 flops is the issue peak in
//                warp instructions per second
//   FP64 FMA     k_peak_dfma: the same with fma on doubles
//   TF32 MMA     k_peak_mma_tf32: one block per SM, one thread issuing
//                tcgen05.mma.cta_group::1.kind::tf32 (M = 128, N = 256,
//                K = 8, A and B in shared memory, accumulator in TMEM) back
//                to back; the kind the six-level tiles use
//
// The paper has no counterpart: these rates only scale the measured kernel
// times against the machine.  Every wait is bounded; on timeout the MMA
// kernel raises its flag and still frees its TMEM.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/mbs.h"
#include "mbs_internal.h"

namespace {

__global__ void __launch_bounds__(256) k_peak_ffma(float *out, int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = 1e-3f * (float)threadIdx.x + (float)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_dfma(double *out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = 1e-3 * (double)threadIdx.x + (double)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ---------------------------------------------------------- tcgen05, TF32
constexpr int MM_M = 128, MM_N = 256, MM_K = 8;              // one MMA
constexpr uint32_t MM_A_BYTES = MM_M * MM_K * 4;              // 4 KB
constexpr uint32_t MM_B_BYTES = MM_N * MM_K * 4;              // 8 KB
constexpr uint32_t MM_SMEM = 96 * 1024;                       // one block per SM
constexpr uint32_t MM_OFF_BAR = MM_A_BYTES + MM_B_BYTES;      // mbarrier, then the TMEM slot

__device__ __forceinline__ uint32_t s_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major operand without swizzle: 8-row x 16-byte core matrices; the two
// K-halves (4 TF32 each) of a row LBO bytes apart, 8-row groups SBO apart;
// descriptor version bits 46-48 = 0b001
__device__ __forceinline__ uint64_t mm_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// kind::tf32 instruction descriptor: D F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9 and 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t mm_idesc(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ uint64_t mm_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mm_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}

// n_mma MMAs of 128 x 256 x 8 into one TMEM accumulator; flag[0] |= 1 if
// the wait for their completion gave up (after 4 s)
__global__ void __launch_bounds__(128, 1) k_peak_mma_tf32(long long n_mma, int *flag, float *sink) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x;
  float *fa = reinterpret_cast<float *>(smem);
  for (int i = tid; i < (int)((MM_A_BYTES + MM_B_BYTES) / 4); i += blockDim.x)
    fa[i] = __uint_as_float(0x3F800000u + ((uint32_t)(i * 2654435761u) & 0x007FE000u));   // TF32 values in [1, 2)
  const uint32_t bar = s_u32(smem + MM_OFF_BAR);
  uint32_t *slot = reinterpret_cast<uint32_t *>(smem + MM_OFF_BAR + 8);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(slot)),
                 "r"((uint32_t)MM_N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *slot;
  bool ok = true;
  if (tid == 0) {
    const uint64_t da = mm_desc(s_u32(smem), MM_M * 16, 128);
    const uint64_t db = mm_desc(s_u32(smem + MM_A_BYTES), MM_N * 16, 128);
    constexpr uint32_t ID = mm_idesc(MM_M, MM_N);
    for (long long k = 0; k < n_mma; ++k) {
      const uint32_t acc = k > 0 ? 1u : 0u;
      asm volatile(
          "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
          "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
          "l"(da), "l"(db), "r"(ID), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
    const uint64_t t0 = mm_ns();
    while (!mm_try_wait(bar, 0))
      if (mm_ns() - t0 > 4000000000ull) {
        ok = false;
        break;
      }
    if (!ok) {
      atomicOr(flag, 1);
      const uint64_t t1 = mm_ns();   // one more bounded wait for the MMAs still in flight
      while (!mm_try_wait(bar, 0) && mm_ns() - t1 < 1000000000ull) {
      }
    }
  }
  __shared__ int s_ok;
  if (tid == 0) s_ok = ok ? 1 : 0;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  ok = s_ok != 0;   // block-uniform
  if (tid < 32) {
    // one accumulator word per block keeps the work observable
    uint32_t v = 0;
    if (ok) {
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(tmem));
      asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(v)::"memory");
    }
    if (tid == 0) sink[blockIdx.x] = __uint_as_float(v);
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)MM_N)
                 : "memory");
  }
}

// Time one launch of `launch` (which enqueues it on stream st) with CUDA events.
template <class F>
cudaError_t timed(cudaStream_t st, F launch, float *ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  if (e == cudaSuccess) {
    launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e;
}

}  // namespace

extern "C" int mbs_peak_rates(int which, double *rate, double *seconds, void *cuda_stream) {
  if (!rate || which < 0 || which > 2) return mbs::set_error(MBS_E_INVALID, "which must be 0 (FP32 FMA), 1 (FP64 FMA) or 2 (TF32 MMA)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return mbs::set_error(MBS_E_CUDA, cudaGetErrorString(e));
  float ms = 0.0f;
  double flops = 0.0;
  void *buf = nullptr;
  int *flag = nullptr;
  if (which <= 1) {
    const int bs = 256, gs = 8 * n_sm;
    const int iters = which == 0 ? 4096 : 256;
    e = cudaMalloc(&buf, (size_t)gs * bs * sizeof(double));
    if (e != cudaSuccess) return mbs::set_error(MBS_E_OOM, cudaGetErrorString(e));
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {   // the last of three (the first ones warm up)
      if (which == 0)
        e = timed(st, [&] { k_peak_ffma<<<gs, bs, 0, st>>>((float *)buf, iters, 0.9999999f, 1e-7f); }, &ms);
      else
        e = timed(st, [&] { k_peak_dfma<<<gs, bs, 0, st>>>((double *)buf, iters, 0.9999999, 1e-7); }, &ms);
    }
    flops = 2.0 * gs * bs * 8.0 * (which == 0 ? 16.0 : 4.0) * iters;
  } else {
    const long long n_mma = 1 << 16;   // ~5 ms at the nominal rate
    e = cudaMalloc(&buf, (size_t)n_sm * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_peak_mma_tf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MM_SMEM);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep)
      e = timed(st, [&] { k_peak_mma_tf32<<<n_sm, 128, MM_SMEM, st>>>(n_mma, flag, (float *)buf); }, &ms);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h) {
      cudaFree(buf);
      cudaFree(flag);
      return mbs::set_error(MBS_E_TIMEOUT, "the tensor-core peak kernel's bounded wait gave up");
    }
    flops = 2.0 * MM_M * MM_N * MM_K * (double)n_mma * n_sm;
  }
  if (buf) cudaFree(buf);
  if (flag) cudaFree(flag);
  if (e != cudaSuccess) return mbs::set_error(MBS_E_CUDA, cudaGetErrorString(e));
  *rate = flops / (ms * 1e-3);
  if (seconds) *seconds = ms * 1e-3;
  return MBS_OK;
}
