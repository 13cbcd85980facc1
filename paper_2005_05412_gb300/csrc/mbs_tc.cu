// mbs_tc.cu -- temporally tiled step for media with N >= 4 levels, the
// constant propagator applied on the fifth-generation tensor cores.
//
// For N levels the Bloch deviation has K = N^2 - 1 components, and the
// constant half of the Strang step (Sec. 2.2, exp(L0 dt) with H0 and the
// Lindblad relaxation) is a dense K x K affine map -- 1,225 multiply-adds per
// cell and step at N = 6, against ~150 for everything else a cell does.  This
// kernel gives that contraction to tcgen05:
//
//   * a block of 128 threads owns one 128-cell tile (thread = cell = MMA row
//     = TMEM lane) and advances it T steps per launch, with the same light-
//     cone halo recompute, float-float fields and warp-edge exchange as the
//     N = 2, 3 tiles (mbs_device.cuh);
//   * per step each thread rotates its cell's coherences by the field angle
//     (the exp(-i mu E dt) factor, exact in the mu eigenbasis) and writes the
//     rotated deviation, augmented by a constant 1, to shared memory as two
//     TF32 operands u = u_hi + u_lo (K-major, no swizzle);
//   * one thread issues D += u_lo W_hi^T + u_hi W_lo^T + u_hi W_hi^T
//     (3xTF32, FP32 accumulation in TMEM; M = 128 cells, N = outputs padded to
//     16, K = inputs padded to 8) onto D seeded by the threads with the
//     rotation increments.  W = [[A - I, c], [w, w0]] so that the MMA also
//     forms the affine offset and the coupling w . u + w0 that drives E;
//   * the threads read their row back (tcgen05.ld), add the whole increment
//     to the deviation with Kahan compensation, and finish the field update.
//
// The tensor-core error is that of the 3xTF32 split (~2^-21 relative per
// product), below the FP32 rounding of the state that the compensated sums
// already absorb.  Every wait on the tensor core is bounded: on timeout the
// block raises flags[1] (MBS_E_TIMEOUT on the host), frees its TMEM and
// returns.
#include <cstring>

#include "mbs_device.cuh"

namespace mbs {
namespace dev {

template <int N, int G>
struct TcShape {
  static constexpr int K = N * N - 1;                 // deviation components
  static constexpr int P = N * (N - 1) / 2;           // coherence pairs
  static constexpr int NP = N - 1;                    // population components
  // TMEM column of deviation component i is i + SH: every coherence pair
  // (NP + 2p, NP + 2p + 1) then starts on an even column and never straddles
  // a 16-column chunk
  static constexpr int SH = NP & 1;
  static constexpr int KA = (K + 1 + 7) / 8 * 8;      // MMA K: [u, 1] padded to the TF32 K step (8)
  static constexpr int NO = (K + SH + 1 + 15) / 16 * 16;   // MMA N: [0^SH, (A - I) u + c, w . u + w0], padded to 16
  static constexpr int NCH = (K + SH + 15) / 16;      // 16-column chunks holding the K components
  static constexpr int M = 128 * G;                   // cells per tile = threads per block: G MMA row groups of 128
  static constexpr int W = M / 32;                    // warps
  // TMEM columns: accumulator [0, NO) (component i at column i + SH, the
  // coupling at K + SH), Kahan compensation words [C_COL, C_COL + 16 NCH)
  // in the same per-chunk positions.  Each step the threads seed the
  // accumulator with the rotation increments (R - 1) x and the MMA adds the
  // propagator's increment onto them.
  // per row group; group h uses columns [h GCOLS, (h + 1) GCOLS)
  static constexpr int C_COL = NO;
  static constexpr int GCOLS = C_COL + 16 * NCH <= 32 ? 32 : C_COL + 16 * NCH <= 64 ? 64 : 128;
  static constexpr int TCOLS = G * GCOLS;   // a power of 2 for G = 1, 2
  static_assert(C_COL + 16 * NCH <= GCOLS && TCOLS <= 256, "TMEM columns");
  static constexpr int CH = KA / 4;                   // 16-byte chunks per operand row
  // canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
  // K-adjacent core matrices LBO bytes apart, row-adjacent ones SBO apart
  static constexpr uint32_t LBO_A = M * 16, LBO_B = NO * 16, SBO = 128;
  static constexpr uint32_t A_BYTES = M * KA * 4, B_BYTES = NO * KA * 4;
  // constant table (built on the host by tc_weight_table, copied verbatim):
  // B_hi | B_lo in their shared-memory layout | zr[2P] | kap0[N-1], each
  // part padded to whole 16-byte vectors
  static constexpr int ZR4 = (2 * P + 3) / 4 * 4, KP4 = (NP + 3) / 4 * 4;
  static constexpr int TAB = 2 * B_BYTES / 4 + ZR4 + KP4;   // floats
  // dynamic shared memory: A_hi | A_lo | table | edge slots | probe rows,
  // indices | mbarrier, TMEM slot
  static constexpr uint32_t OFF_TAB = 2 * A_BYTES;
  static constexpr uint32_t OFF_ZR = OFF_TAB + 2 * B_BYTES;
  static constexpr uint32_t OFF_KP = OFF_ZR + ZR4 * 4;
  static constexpr uint32_t OFF_X = OFF_TAB + TAB * 4;
  static constexpr uint32_t OFF_PR = OFF_X + W * 16;
  static constexpr uint32_t OFF_PV = OFF_PR + 2 * MAXPROBE * 4;   // E_b^{n-1} of the ends: 4 floats
  static constexpr uint32_t OFF_BAR = OFF_PV + 16;
  static constexpr uint32_t SMEM = OFF_BAR + 16;   // mbarrier (8 bytes), TMEM address, max |kappa_0k|
  static_assert(NCH * 16 <= NO, "compensation chunks fit their columns");
  // chunk of the seeded accumulator after which A chunk c (elements 4c..4c+3
  // of [u, 1, 0...]) is known; -1: populations and constants only
  __host__ __device__ static constexpr int a_step(int c) {
    int st = -1;
    for (int e = 0; e < 4; ++e) {
      const int j = 4 * c + e;
      if (j >= NP && j < K && (j + SH) / 16 > st) st = (j + SH) / 16;
    }
    return st;
  }
};

// ------------------------------------------------------ tcgen05 primitives
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor (tcgen05): start address, leading- and
// stride-dimension byte offsets (all >> 4), fixed version bits 46-48 = 0b001,
// base offset 0, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         ((uint64_t)1 << 46);
}

// instruction descriptor, kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One test of the barrier phase; a thread whose phase is not complete is
// suspended (it issues nothing) until the phase completes or about 0.1 ms
// pass, so that waiting warps leave the issue slots to the other blocks.
__device__ __forceinline__ bool bar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of the barrier, for at most ~1 s; false on timeout.
__device__ __forceinline__ bool bar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (bar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (!bar_try_wait(bar, parity))
    if (global_ns() - t0 > 1000000000ull) return false;
  return true;
}

// 16 consecutive FP32 columns of this thread's TMEM lane; the wait takes the
// registers as operands so that no use is scheduled before the data arrive
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])::"memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// two such loads (columns ta.. and tb..) under one wait
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, float (&va)[16], uint32_t tb, float (&vb)[16]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(ta));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(tb));
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                 "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                 "+r"(r[29]), "+r"(r[30]), "+r"(r[31])::"memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    va[i] = __uint_as_float(r[i]);
    vb[i] = __uint_as_float(r[16 + i]);
  }
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// round to TF32 (10 explicit mantissa bits, nearest, ties away from zero) by
// integer arithmetic on the bits: two integer operations that the compiler
// folds for constant operands
__device__ __forceinline__ float to_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void sts128(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

// rho probes of warp `wib`'s cells: for each list entry (rows | index + 256
// quantity, build_probe_list) that is a rho probe of this warp, the warp
// evaluates the functional together (lane l takes terms l, l + 32) from the
// probe cell's operand row, u = hi + lo exactly, with the row's constant 1 at
// element K.  Out of line: only warps that hold a probe call it, and its
// registers stay out of the step's allocation.
template <int K, uint32_t LBO_A, uint32_t A_BYTES>
static __device__ __noinline__ void rho_probes_warp(const int *s_plr, const int *s_plp, const unsigned char *smem,
                                                    const float *pcoef, float *rec, long long nt, long long n,
                                                    int wib, int lane) {
  __syncwarp();   // the warp's operand rows are written
  for (int k = 0; k < MAXPROBE; ++k) {
    const int r = s_plr[k];
    if (r < 0) break;
    if ((r >> 5) != wib || s_plp[k] < 512) continue;
    const int p = s_plp[k] & 255;
    const float *cf = pcoef + (size_t)p * (K + 1);
    float v = 0.0f;
    for (int i = lane; i <= K; i += 32) {
      const uint32_t off = (uint32_t)(i >> 2) * LBO_A + (uint32_t)r * 16 + (uint32_t)(i & 3) * 4;
      v = fmaf(cf[i], *reinterpret_cast<const float *>(smem + off) + *reinterpret_cast<const float *>(smem + A_BYTES + off),
               v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if (lane == 0) rec[(size_t)p * nt + n] = v;
  }
}

// ---------------------------------------------------------------- kernel
// Tile b owns cells [b*own, (b+1)*own), own = 128 - 2T; thread i holds cell
// tb + i with tb = b*own - T (the tile holding the last cell may start 4 or 8
// cells earlier, as in the N = 2, 3 tiles).  Requires one medium parameter
// slot (slot 0) and no per-cell operators.  Reads buffers `cur`, writes the
// owned cells of buffers cur ^ 1.
//
// Per thread the deviation lives in registers and its Kahan compensation in
// the thread's TMEM lane, which keeps the block at <= 128 registers per
// thread: four blocks (16 warps) per SM.
template <int N, int G>
__global__ void __launch_bounds__(128 * G, 4 / G)
    k_tiled_tc(const __grid_constant__ Args a, long long n0, int nsteps, int T, int cur) {
  using S = TcShape<N, G>;
  constexpr int K = S::K, P = S::P, NP = S::NP, SH = S::SH;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, wib = tid >> 5;
  const int own = S::M - 2 * T;
  const int c_own = blockIdx.x * own;
  if (c_own >= a.nx) return;   // the whole block leaves together
  if (*a.flags != 0) return;   // a state check failed: the solve stops (before any TMEM is held)

  const uint32_t sA_hi = smem_u32(smem), sA_lo = sA_hi + S::A_BYTES;
  const uint32_t sB_hi = sA_lo + S::A_BYTES, sB_lo = sB_hi + S::B_BYTES;
  const float *s_zr = reinterpret_cast<const float *>(smem + S::OFF_ZR);   // zr[2P]
  // the probes of this tile's owned cells (build_probe_list, keyed by tile
  // row = thread)
  int *s_plr = reinterpret_cast<int *>(smem + S::OFF_PR);
  int *s_plp = s_plr + MAXPROBE;
  float *s_x = reinterpret_cast<float *>(smem + S::OFF_X);     // [warp][E hi, E lo, H hi, H lo]
  const uint32_t bar = smem_u32(smem + S::OFF_BAR);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(smem + S::OFF_BAR + 8);

  // ---- constant table: weights W (rows = outputs; row i + SH =
  // [(A - I)_i., c_i], row K + SH = [w, w0], other rows 0) as TF32 hi/lo,
  // reference coherences, field angles of the pairs (0, k); probe tables
  {
    const float4 *src = reinterpret_cast<const float4 *>(a.tcw);
    float4 *dst = reinterpret_cast<float4 *>(smem + S::OFF_TAB);
#pragma unroll
    for (int r = 0; r < (S::TAB / 4 + S::M - 1) / S::M; ++r) {
      const int i = tid + r * S::M;
      if (i < S::TAB / 4) dst[i] = src[i];
    }
  }
  fence_async_smem();
  if (tid == 0) bar_init(bar, 1);
  if (wib == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"((uint32_t)S::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }

  // ---- tile geometry and this thread's cell
  int tb = c_own - T;
  if (a.nx - 1 < c_own + own) {
    if (a.nx - 1 == c_own || (a.nx - 1 - tb) % 32 == 0) tb -= 4;
    if ((a.nx - 1 - tb) % 32 == 0) tb -= 4;
  }
  const int lo = c_own - tb;      // tile position of the first owned cell
  const int g0 = tb + tid;        // this thread's cell
  const int base = a.off + g0;    // its array index (>= 0)

  float E = reinterpret_cast<const float *>(a.E[cur])[base];
  float El = reinterpret_cast<const float *>(a.El[cur])[base];
  float H = reinterpret_cast<const float *>(a.H[cur])[base];
  float Hl = reinterpret_cast<const float *>(a.Hl[cur])[base];
  float d[K];
  {
    const float *Din = reinterpret_cast<const float *>(a.D[cur]);
#pragma unroll
    for (int i = 0; i < K; ++i) d[i] = Din[(size_t)i * a.ld + base];
  }
  const float *emc = reinterpret_cast<const float *>(a.emc);
  const int mt = a.mat[base];
  const float ca = emc[mt * 4 + 0], cb = emc[mt * 4 + 1];
  const float ch = g0 == 0 ? 0.0f : emc[mt * 4 + 2];   // face 0 is a fixed boundary slot
  const float mk = a.qslot[mt] >= 0 ? 1.0f : 0.0f;

  const int t_lo = tb + wib * 32, t_hi = t_lo + 32;   // this warp's cells
  bool any_src = false;
  for (int s = 0; s < a.n_src; ++s)
    any_src |= (a.src[s].cell >= t_lo && a.src[s].cell < t_hi) || (a.src[s].face >= t_lo && a.src[s].face < t_hi);
  const bool any_bnd = (t_lo <= 0 && 0 < t_hi) || (t_lo <= a.nx - 1 && a.nx - 1 < t_hi);
  const bool owned = tid >= lo && tid < lo + own && tid < S::M - T;
  float *rec = reinterpret_cast<float *>(a.rec);
  const float *pcoef = reinterpret_cast<const float *>(a.pr_coef);

  // E_b^{n-1} of the two ends (partially reflecting ends), from the previous
  // launch; kept in shared memory (only the lanes holding an end use it)
  float *s_pv = reinterpret_cast<float *>(smem + S::OFF_PV);   // left hi, lo, right hi, lo
  if (tid < 4) s_pv[tid] = reinterpret_cast<const float *>(a.bprev[cur])[tid];
  build_probe_list(a, [&](int c) {
    const int r = c - tb;   // tile row of the probe cell
    return r >= lo && r < lo + own && r < S::M - T ? r : -1;
  }, s_plr, s_plp);
  if (lane == 31) {
    s_x[wib * 4 + 0] = E;
    s_x[wib * 4 + 1] = El;
  }
  // largest |kappa_0k|: |theta_0k| <= |E| kap_max (kept in shared memory:
  // registers are full)
  float *s_kmax = reinterpret_cast<float *>(smem + S::OFF_BAR + 12);
  if (tid == 0) {
    const float *kp = reinterpret_cast<const float *>(a.tcw) + (S::OFF_KP - S::OFF_TAB) / 4;
    float m = 0.0f;
    for (int k = 0; k < NP; ++k) m = fmaxf(m, fabsf(kp[k]));
    *s_kmax = m;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  bool probe = false;
  for (int k = 0; k < MAXPROBE && s_plr[k] >= 0; ++k) probe |= s_plr[k] == tid;
  const bool warp_probe = __any_sync(FULL, probe);   // some cell of the warp is a probe cell
  // field angles of the pairs (0, k), k = 1..N-1; every other pair's angle
  // is a difference of two of them (theta_jk = theta_0k - theta_0j)
  const float *kap0 = reinterpret_cast<const float *>(smem + S::OFF_KP);
  // this warp's TMEM lanes (warp w reaches lanes 32 (w mod 4) ..) in its row group's columns
  const uint32_t t_row = tmem + ((uint32_t)((wib & 3) * 32) << 16) + (uint32_t)((wib >> 2) * S::GCOLS);
  const uint32_t t_cmp = t_row + S::C_COL;                        // its compensation words
  {
    // compensation words of the cell into TMEM (column i + SH)
    const float *Cin = reinterpret_cast<const float *>(a.C[cur]);
#pragma unroll
    for (int c16 = 0; c16 < S::NCH; ++c16) {
      float v[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int i = 16 * c16 + e - SH;
        v[e] = (i >= 0 && i < K) ? Cin[(size_t)i * a.ld + base] : 0.0f;
      }
      tmem_st16(t_cmp + 16 * c16, v);
    }
    tmem_wait_st();
  }
  constexpr uint32_t IDESC = idesc_tf32(128, S::NO);
  uint32_t phase = 0;
  bool timed_out = false;   // this thread's wait gave up
  int stop = 0;             // some thread's wait gave up (block-uniform)

  // A operand chunk c of this cell's row: [u, 1, 0...] elements 4c..4c+3 as
  // TF32 hi and lo.  hi = u rounded to TF32; lo = u - hi is exact in FP32 and
  // goes to the tensor core unrounded: the MMA uses its leading 19 bits, so
  // the operand pair represents u to 2^-21 relative (2^-22 if rounded).
  // (Passing u itself as hi, for the tensor core to shorten, is not
  // equivalent: measured, it moves the six-level traces by 4e-4.)
  auto put_a = [&](int c, const float (&u)[K]) {
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = 4 * c + e;
      const float v = j < K ? u[j] : (j == K ? 1.0f : 0.0f);
      h[e] = to_tf32(v);
      l[e] = v - h[e];
    }
    const uint32_t off = (uint32_t)c * S::LBO_A + (uint32_t)tid * 16;
    sts128(sA_hi + off, h[0], h[1], h[2], h[3]);
    sts128(sA_lo + off, l[0], l[1], l[2], l[3]);
  };

#pragma unroll 1
  for (int t = 0; t < nsteps; ++t) {
    const long long n = n0 + t;
    // ---- H^{n+1/2} on the left face of the cell
    {
      float elh = __shfl_up_sync(FULL, E, 1), ell = __shfl_up_sync(FULL, El, 1);
      if (lane == 0 && wib > 0) {
        elh = s_x[(wib - 1) * 4 + 0];
        ell = s_x[(wib - 1) * 4 + 1];
      }
      fld_axpy_diff<float, true>(H, Hl, ch, E, El, elh, ell, -0.0f);   // -0: the extra addition drops out
    }
    if (any_src)
      for (int s = 0; s < a.n_src; ++s)
        if (a.src[s].face == g0) {
          float vh, vl;
          src_val<float>(a.src[s].sH, n, a.nt, vh, vl);
          fld_add<float>(H, Hl, vh, vl);
        }
    if (lane == 0) {
      s_x[wib * 4 + 2] = H;
      s_x[wib * 4 + 3] = Hl;
    }
    // ---- field rotation, u = delta + (R - 1) x; the increments (R - 1) x
    // seed the accumulator, the MMA adds (A - I) u + c to them
    {
      const float ej = fld_val<float>(E, El) * mk;
      float sn[N], cm[N];   // sin, cos - 1 of theta_0k (k = 0: zero angle)
      sn[0] = cm[0] = 0.0f;
      // the shorter polynomials, exact to 2 and 3 ulp while |theta_0k| <= 1/2;
      // larger angles take the library routine below
#pragma unroll
      for (int k = 1; k < N; ++k) sincos_m1_taylor_half(kap0[k - 1] * ej, sn[k], cm[k]);
      if (__any_sync(FULL, fabsf(ej) * *s_kmax > 0.5f))   // a strong field somewhere in the warp
        for (int k = 1; k < N; ++k)
          if (fabsf(kap0[k - 1] * ej) > 0.5f) {
            const float2 r = sincos_m1_far(kap0[k - 1] * ej);
            sn[k] = r.x;
            cm[k] = r.y;
          }
      float u[K];
#pragma unroll
      for (int i = 0; i < NP; ++i) u[i] = d[i];
#pragma unroll
      for (int c = 0; c < S::CH; ++c)
        if (S::a_step(c) < 0) put_a(c, u);
#pragma unroll
      for (int c16 = 0; c16 < S::NO / 16; ++c16) {
        float seed[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) seed[e] = 0.0f;
#pragma unroll
        for (int e = 0; e < 16; e += 2) {
          const int i = 16 * c16 + e - SH;   // first component of a pair?
          if (i < NP || i >= K) continue;
          const int pr = (i - NP) / 2;
          int j = 0, k = 0;                  // the pair's levels
          for (int jj = 0, q2 = 0; jj < N; ++jj)
            for (int kk = jj + 1; kk < N; ++kk, ++q2)
              if (q2 == pr) { j = jj; k = kk; }
          float sv, mv;
          if (j == 0) {
            sv = sn[k];
            mv = cm[k];
          } else {   // sin, cos - 1 of theta_0k - theta_0j
            sv = (sn[k] - sn[j]) + fmaf(sn[k], cm[j], -(cm[k] * sn[j]));
            mv = fmaf(cm[k], cm[j], fmaf(sn[k], sn[j], cm[k] + cm[j]));
          }
          const float2 z = reinterpret_cast<const float2 *>(s_zr)[pr];
          const float xa = z.x + d[i], xb = z.y + d[i + 1];
          const float ra = mv * xa - sv * xb;
          const float rb = sv * xa + mv * xb;
          u[i] = d[i] + ra;
          u[i + 1] = d[i + 1] + rb;
          seed[e] = ra;
          seed[e + 1] = rb;
        }
        tmem_st16(t_row + 16 * c16, seed);
#pragma unroll
        for (int c = 0; c < S::CH; ++c)
          if (S::a_step(c) == c16) put_a(c, u);
      }
    }
    tmem_wait_st();
    fence_async_smem();
    if (warp_probe)
      rho_probes_warp<K, S::LBO_A, S::A_BYTES>(s_plr, s_plp, smem, pcoef, rec, a.nt, n, wib, lane);
    tc_fence_before();
    __syncthreads();   // operands written; H of the warp edges published
    if (tid == 0 && !a.test_stall) {
      tc_fence_after();
      const uint64_t dA_hi = umma_desc(sA_hi, S::LBO_A, S::SBO), dA_lo = umma_desc(sA_lo, S::LBO_A, S::SBO);
      const uint64_t dB_hi = umma_desc(sB_hi, S::LBO_B, S::SBO), dB_lo = umma_desc(sB_lo, S::LBO_B, S::SBO);
#pragma unroll
      for (int h = 0; h < G; ++h) {   // row group h: rows 128 h.., 16 row groups of 8 further in A
        const uint32_t d = tmem + (uint32_t)(h * S::GCOLS);
#pragma unroll
        for (int k = 0; k < S::KA / 8; ++k) {
          const uint64_t oa = (uint64_t)((2 * k * S::LBO_A + h * 16 * S::SBO) >> 4);
          const uint64_t ob = (uint64_t)((2 * k * S::LBO_B) >> 4);
          mma_tf32(d, dA_lo + oa, dB_hi + ob, IDESC, 1u);
          mma_tf32(d, dA_hi + oa, dB_lo + ob, IDESC, 1u);
          mma_tf32(d, dA_hi + oa, dB_hi + ob, IDESC, 1u);
        }
      }
      mma_commit(bar);
    }
    timed_out |= !bar_wait_bounded(bar, phase);
    phase ^= 1u;
    tc_fence_after();
    // ---- delta += (R - 1) x + (A - I) u + c (compensated); coupling w . u + w0
    float pw = 0.0f;
#pragma unroll
    for (int c16 = 0; c16 < S::NO / 16; ++c16) {
      if (16 * c16 > K + SH) break;
      float acc[16], cw[16];
      if (c16 < S::NCH)
        tmem_ld16x2(t_row + 16 * c16, acc, t_cmp + 16 * c16, cw);
      else
        tmem_ld16(t_row + 16 * c16, acc);
      if (c16 < S::NCH) {
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const int i = 16 * c16 + e - SH;
          if (i >= 0 && i < K) kahan_add(d[i], cw[e], acc[e]);
        }
        tmem_st16(t_cmp + 16 * c16, cw);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e)
        if (16 * c16 + e - SH == K) pw = acc[e] * mk;
    }
    // ---- boundary cells: keep E^n of the boundary cell and its neighbour
    float bo_h = 0.0f, bo_l = 0.0f, no_h = 0.0f, no_l = 0.0f;
    if (any_bnd) {
      const float r_oh = __shfl_down_sync(FULL, E, 1), r_ol = __shfl_down_sync(FULL, El, 1);
      const float l_oh = __shfl_up_sync(FULL, E, 1), l_ol = __shfl_up_sync(FULL, El, 1);
      if (g0 == 0) {
        bo_h = E; bo_l = El; no_h = r_oh; no_l = r_ol;
      }
      if (g0 == a.nx - 1) {
        bo_h = E; bo_l = El; no_h = l_oh; no_l = l_ol;
      }
    }
    // ---- E^{n+1}
    {
      float hrh = __shfl_down_sync(FULL, H, 1), hrl = __shfl_down_sync(FULL, Hl, 1);
      if (lane == 31 && wib < S::W - 1) {
        hrh = s_x[(wib + 1) * 4 + 2];
        hrl = s_x[(wib + 1) * 4 + 3];
      }
      fld_axpy_diff<float, true>(E, El, cb, hrh, hrl, H, Hl, ca * fld_val<float>(E, El) - pw);
    }
    if (any_src)
      for (int s = 0; s < a.n_src; ++s)
        if (a.src[s].cell == g0) {
          float vh, vl;
          src_val<float>(a.src[s].sE, n, a.nt, vh, vl);
          if (a.src[s].kind == 2) {
            E = vh;
            El = vl;
          } else {
            fld_add<float>(E, El, vh, vl);
          }
        }
    if (any_bnd) {
      // E_b^{n+1} = E_nb^n + k (E_nb^{n+1} - E_b^n), or 0 for a mirror
      const float r_nh = __shfl_down_sync(FULL, E, 1), r_nl = __shfl_down_sync(FULL, El, 1);
      const float l_nh = __shfl_up_sync(FULL, E, 1), l_nl = __shfl_up_sync(FULL, El, 1);
      const bool lft = g0 == 0, rgt = g0 == a.nx - 1;
      if (lft || rgt) {
        const float nh = lft ? r_nh : l_nh, nl = lft ? r_nl : l_nl;
        const int bc = lft ? a.bc_l : a.bc_r;
        if (bc == 1) {
          E = El = 0.0f;
        } else {
          float bh = no_h, bl = no_l;
          fld_axpy_diff<float>(bh, bl, float(lft ? a.kmur_l : a.kmur_r), nh, nl, bo_h, bo_l, 0.0f);
          if (bc == 2) partial_reflect<float>(bh, bl, float(lft ? a.r_l : a.r_r), s_pv[lft ? 0 : 2], s_pv[lft ? 1 : 3]);
          E = bh;
          El = bl;
        }
        s_pv[lft ? 0 : 2] = bo_h;   // E_b^n becomes the next step's E_b^{n-1}
        s_pv[lft ? 1 : 3] = bo_l;
      }
    }
    if (probe)
      for (int k = 0; k < MAXPROBE && s_plr[k] >= 0; ++k)
        if (s_plr[k] == tid && s_plp[k] < 512)
          rec[(size_t)(s_plp[k] & 255) * a.nt + n] = s_plp[k] < 256 ? fld_val<float>(E, El) : fld_val<float>(H, Hl);
    if (lane == 31) {
      s_x[wib * 4 + 0] = E;
      s_x[wib * 4 + 1] = El;
    }
    tmem_wait_st();
    tc_fence_before();
    stop = __syncthreads_or(timed_out);   // E of the warp edges published
    if (stop) {
      if (tid == 0) atomicOr(a.flags + 1, 1);
      break;
    }
  }

  // ---- compensation words back from TMEM, then release it (after a last
  // bounded wait if a step gave up)
  float cc[K];
#pragma unroll
  for (int c16 = 0; c16 < S::NCH; ++c16) {
    float cw[16];
    tmem_ld16(t_cmp + 16 * c16, cw);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int i = 16 * c16 + e - SH;
      if (i >= 0 && i < K) cc[i] = cw[e];
    }
  }
  if (stop && tid == 0) bar_wait_bounded(bar, phase ^ 1u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (wib == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)S::TCOLS)
                 : "memory");

  // ---- write back the owned cells
  if (!owned || g0 >= a.nx) return;
  if (g0 == 0 || g0 == a.nx - 1) {   // E_b^{n-1} for the next launch
    float *bp = reinterpret_cast<float *>(a.bprev[cur ^ 1]);
    if (g0 == 0) {
      bp[0] = s_pv[0];
      bp[1] = s_pv[1];
    }
    if (g0 == a.nx - 1) {
      bp[2] = s_pv[2];
      bp[3] = s_pv[3];
    }
  }
  ff_renorm(E, El);
  ff_renorm(H, Hl);
  reinterpret_cast<float *>(a.E[cur ^ 1])[base] = E;
  reinterpret_cast<float *>(a.El[cur ^ 1])[base] = El;
  reinterpret_cast<float *>(a.H[cur ^ 1])[base] = H;
  reinterpret_cast<float *>(a.Hl[cur ^ 1])[base] = Hl;
  float *Do = reinterpret_cast<float *>(a.D[cur ^ 1]);
  float *Co = reinterpret_cast<float *>(a.C[cur ^ 1]);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    Do[(size_t)i * a.ld + base] = d[i];
    Co[(size_t)i * a.ld + base] = cc[i];
  }
}

template <int N, int G>
int tiled_tc_impl(const Args &a, long long n0, int nsteps, int T, int cur, cudaStream_t st) {
  using S = TcShape<N, G>;
  static_assert(S::M - 5 <= PAD, "a tile reaches past the pad cells");
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev < 0 || dev >= 64) return (int)cudaErrorInvalidDevice;
  if (!attr_set[dev]) {
    e = cudaFuncSetAttribute(k_tiled_tc<N, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (e == cudaSuccess)   // all of the unified L1/shared storage as shared memory
      e = cudaFuncSetAttribute(k_tiled_tc<N, G>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return (int)e;
    attr_set[dev] = true;
  }
  const int own = S::M - 2 * T;
  const int gs = (a.nx + own - 1) / own;
  k_tiled_tc<N, G><<<gs, S::M, S::SMEM, st>>>(a, n0, nsteps, T, cur);
  return (int)cudaGetLastError();
}

}  // namespace dev

namespace {
// round to TF32: nearest, ties away from zero (10 explicit mantissa bits)
float tf32_host(float x) {
  uint32_t b;
  std::memcpy(&b, &x, 4);
  b = (b + 0x1000u) & 0xFFFFE000u;
  float y;
  std::memcpy(&y, &b, 4);
  return y;
}

template <int N>
int tc_table_impl(const double *qb, float *out) {
  using S = dev::TcShape<N, 1>;
  if (!out) return S::TAB;
  constexpr int K = S::K, P = S::P;
  for (int i = 0; i < S::TAB; ++i) out[i] = 0.0f;
  float *bh = out, *bl = out + S::B_BYTES / 4;
  auto at = [&](int i, int j) { return qb[i * K + j]; };   // (A - I) row-major
  for (int o = 0; o < S::NO; ++o)
    for (int j = 0; j < S::KA; ++j) {
      const int i = o - S::SH;
      double v = 0.0;
      if (i >= 0 && i < K)
        v = j < K ? at(i, j) : (j == K ? qb[K * K + i] : 0.0);
      else if (i == K)
        v = j < K ? qb[K * K + K + j] : (j == K ? qb[K * K + 2 * K] : 0.0);
      const float hi = tf32_host((float)v);
      const float lo = tf32_host((float)(v - (double)hi));
      const int idx = ((j >> 2) * (int)S::LBO_B + o * 16 + (j & 3) * 4) / 4;
      bh[idx] = hi;
      bl[idx] = lo;
    }
  float *zr = out + 2 * S::B_BYTES / 4, *kp = zr + S::ZR4;
  for (int i = 0; i < 2 * P; ++i) zr[i] = (float)qb[K * K + 2 * K + 1 + P + i];
  for (int k = 0; k < S::NP; ++k) kp[k] = (float)qb[K * K + 2 * K + 1 + k];
  return S::TAB;
}
}  // namespace

int tc_weight_table(int N, const double *qblk, float *out) {
  switch (N) {
    case 4: return tc_table_impl<4>(qblk, out);
    case 5: return tc_table_impl<5>(qblk, out);
    case 6: return tc_table_impl<6>(qblk, out);
  }
  return 0;
}

int tiled_tc_supported(int prec, int N) { return prec == 1 && N >= 4 && N <= 6; }

// The kernel's tile placement (as in k_tiled_tc): the tile that owns the
// last cell starts 4 or 8 cells early when the last cell would be its first
// owned cell or start a warp.  T is usable when, for this grid, the last cell
// stays owned with its neighbour in the same warp and inside the light cone,
// and cell 0's neighbour is in the same warp and inside the light cone.
bool tiled_tc_geometry_ok(int nx, int cells, int T) {
  if ((cells != 128 && cells != 256) || T < 1 || cells - 2 * T < 32 || nx < 1) return false;
  const int own = cells - 2 * T;
  auto start = [&](int c_own) {
    int tb = c_own - T;
    if (nx - 1 < c_own + own) {
      if (nx - 1 == c_own || (nx - 1 - tb) % 32 == 0) tb -= 4;
      if ((nx - 1 - tb) % 32 == 0) tb -= 4;
    }
    return tb;
  };
  const int c_last = (nx - 1) / own * own;
  const int p = nx - 1 - start(c_last);          // tile position of the last cell
  if (!(p >= T + 1 && p < cells - T && p % 32 != 0)) return false;
  const int q = -start(0);                       // tile position of cell 0
  return q % 32 != 31 && q + 1 <= cells - 1 - T;
}

int launch_tiled_tc(const Args &a, int cells, long long n0, int nsteps, int T, int cur, void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (a.prec != 1 || a.n_slot != 1 || a.pcell || !a.tcw || a.n_probe > MAXPROBE || !tiled_tc_geometry_ok(a.nx, cells, T))
    return (int)cudaErrorInvalidValue;
  const bool wide = cells == 256;
  switch (a.N) {
    case 4: return wide ? dev::tiled_tc_impl<4, 2>(a, n0, nsteps, T, cur, st) : dev::tiled_tc_impl<4, 1>(a, n0, nsteps, T, cur, st);
    case 5: return wide ? dev::tiled_tc_impl<5, 2>(a, n0, nsteps, T, cur, st) : dev::tiled_tc_impl<5, 1>(a, n0, nsteps, T, cur, st);
    case 6: return wide ? dev::tiled_tc_impl<6, 2>(a, n0, nsteps, T, cur, st) : dev::tiled_tc_impl<6, 1>(a, n0, nsteps, T, cur, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace mbs
