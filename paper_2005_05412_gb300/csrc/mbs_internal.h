// mbs_internal.h -- private interface between the host setup (mbs_host.cpp)
// and the CUDA kernels (mbs_device.cuh, instantiated in mbs_tiled.cu and
// mbs_plain*.cu) of the Maxwell-Bloch hot path.
//
// State representation on the device (per medium cell):
//   * the density matrix after the first half of the constant propagator,
//     x^n = exp(L0 dt/2) rho^{n-1/2}, in real coordinates of the dipole
//     eigenbasis (rho~ = V^+ rho V): populations rho~_kk (k < N-1) and the
//     (Re, Im) pairs of rho~_jk, j < k -- K = N^2 - 1 numbers;
//   * stored as the deviation delta = x - x_ref from a reference state
//     (the steady state of L0 when unique, else the initial state), so that
//     near-unity populations keep their low-order bits in FP32;
//   * in FP32, a Kahan compensation word per component.
// One time step (Strang splitting with adjacent half steps merged):
//   v = R(E^n) x  (exact field propagator: rotation of each coherence pair by
//                  theta_p = kappa_p E^n, populations unchanged)
//   u = v - x_ref = delta + (R - 1) x
//   delta' = A u + c          (A = exp(L0 dt) on deviations, c its offset)
//   d_t P^{n+1/2} = n3D (g . u + g0)  (tr{mu L0 exp(L0 dt/2) v})
//   E^{n+1} = E^n + (a' - 1) E^n - b' Gamma d_t P + b' (H_{m+1} - H_m)/dz
// Fields: E in V/m; H is stored normalised, H^ = eta0 H (V/m), so that in
// vacuum at Courant number 1 both field coefficients are exactly 1.  In FP32
// each field value is a float-float pair (high + low word).
#pragma once
#include <cstddef>
#include <cstdint>
#include <vector_types.h>

namespace mbs {

constexpr int NMAX = 6;
constexpr int MAXSRC = 4;
constexpr int MAXPROBE = 64;
constexpr int PAD = 512;  // left/right margin cells of every cell array

// Tiled kernel geometry per level count (the fastest measured on GB300): a
// block of W warps advances one contiguous tile of 32 W R cells (R cells per
// lane) by T steps and owns the tile minus a T-cell halo on each side.
// T <= 32 R - 12 leaves room for the shift of the tile that holds the
// absorbing right end (at most 8 cells).
template <int N>
struct TileGeom {
  static constexpr int R = N == 2 ? 4 : 2;
  static constexpr int W = N == 2 ? 4 : 8;
};
inline int tile_lane_cells(int N) { return N == 2 ? TileGeom<2>::R : TileGeom<3>::R; }
inline int tile_warps(int N) { return N == 2 ? TileGeom<2>::W : TileGeom<3>::W; }
inline int tile_own(int N, int T) { return 32 * tile_warps(N) * tile_lane_cells(N) - 2 * T; }
inline int tile_max_steps(int N) { return 32 * tile_lane_cells(N) - 12; }

// Packed per-quantum-material parameter block (in the state's real type):
//   am1[K*K] (A - I, row-major) | c[K] | w[K] | w0 | kap[P] | zr[2P]
// w, w0 already include b' Gamma n3D, i.e. E -= w . u + w0 [V/m].
inline int q_k(int N) { return N * N - 1; }
inline int q_p(int N) { return N * (N - 1) / 2; }
inline int q_stride(int N) {
  int K = q_k(N), P = q_p(N);
  return (K * K + 2 * K + 1 + 3 * P + 3) / 4 * 4;   // 16-byte multiple in FP32 (rows load as vectors)
}
// Per-cell parameter rows (cells with their own propagator): am1, c, w, w0.
inline int pc_rows(int N) {
  int K = q_k(N);
  return K * K + 2 * K + 1;
}

struct SrcDev {
  int kind;         // 0 TF/SF +x, 1 TF/SF -x, 2 hard
  int face;         // face receiving the H correction (-1: none)
  int cell;         // cell receiving the E correction / hard value
  int pad_;
  const void *sH;   // H^ correction per step (added at `face`): FP64 [nt],
                    // FP32 [2][nt] (high words, then low words)
  const void *sE;   // E correction (or hard value) per step, same layout
};

// Everything a launch needs (passed by value).
struct Args {
  int prec;                    // 0 = FP64, 1 = FP32
  int N, K, P;
  int nx, ld, off;             // cells, padded row length, index of cell 0
  long long nt;                // total steps of the scenario
  void *E[2], *H[2];           // [ld] ping-pong (plain path updates H in place in H[0])
  void *El[2], *Hl[2];         // FP32: low words of the float-float fields (else null)
  void *D[2], *C[2];           // [K][ld] deviation / Kahan compensation
  void *pd;                    // [ld] coupling term of the plain path
  const uint8_t *mat;          // [ld] material id per cell (pad cells: n_mat)
  int n_mat_all;               // materials incl. the pad material
  const void *emc;             // [n_mat_all][4]: a' - 1, b^, c^, 0
  const int *qslot;            // [n_mat_all]: parameter slot or -1
  const void *qpar;            // [n_slot][qstride]
  int n_slot, qstride;
  const void *pcell;           // [pc_rows][ld] per-cell parameters or null
  const void *pcell2;          // [7][ld] structured two-level rows (see PrmBloch2) or null

  int n_src;
  SrcDev src[MAXSRC];
  int bc_l, bc_r;              // 0 = Mur, 1 = PEC, 2 = partially reflecting
  double kmur_l, kmur_r;
  double r_l, r_r;             // amplitude reflections -sqrt(R) (bc 2)
  void *bprev[2];              // ping-pong [left hi, left lo, right hi, right lo]: E_b^{n0-1}
  int n_probe;
  const int *pr_cell;          // [n_probe]
  const int *pr_q;             // [n_probe] quantity
  const void *pr_coef;         // [n_probe][K+1]: rho probes h_K, h0
  const float *tcw;            // tensor-core tiles: weight table (tc_weight_table) or null
  void *rec;                   // [n_probe][nt]
  const double *zref;          // [n_slot][N*N] reference states (full real coordinates, FP64)
  int *flags;                  // [4] device status words: [0] bit 0 a non-finite value, bit 1 a state that
                               // is not a density matrix (beyond the tolerance); any bit set makes every
                               // later step launch of the scenario return at once; [1] a bounded wait gave up
  int test_stall;              // test of the failure path: the tensor-core tiles issue no MMA, so their
                               // first bounded wait expires (about 1 s) and the solve reports a timeout
};

// Batched single-cell solver (mbs_cells.cu): one thread per driven system.
struct CellsArgs {
  int prec, N, n_sys;
  long long nt;
  int every;               // record every `every` steps
  const void *prm;         // [rows][n_sys]: A - I | c | kap | zr | population functionals
  void *D, *C;             // [K][n_sys] deviation / Kahan compensation (updated in place)
  const void *amp;         // [n_sys] drive amplitude
  const int *tab_id;       // [n_sys] drive shape
  const void *tab;         // drive shapes: FP64 [n_tab][nt]; FP32 [n_tab][2][nt] (high, low words)
  long long tab_stride;    // reals per shape
  void *rec;               // [n_rec][N][n_sys] populations
  const double *zref;      // [n_sys][N*N] reference states (full real coordinates)
  int *flags;              // [4]
};
int launch_cells(const CellsArgs &a, long long n0, int nsteps, void *stream);
int launch_cells_check(const CellsArgs &a, double *min_eig, double *tr_dev, void *stream);

// Records `msg` as the calling thread's last error (mbs_last_error) and
// returns `code` (mbs_host.cpp).
int set_error(int code, const char *msg);

// Launchers (mbs_tiled.cu, mbs_plain.cu).  All return 0 or a cudaError_t value.
int launch_plain_step(const Args &a, long long n, int cur, void *stream);
int launch_tiled(const Args &a, long long n0, int nsteps, int T, int cur, void *stream);
int tiled_supported(int prec, int N);
int tiled_variant(const Args &a);
size_t tiled_batch_smem(int prec, int N, int max_mat_all, int max_slot, int max_qstride);
int launch_tiled_batch(int prec, int N, int pm, const Args *args, const int2 *tasks, int n_tasks, size_t smem,
                       long long n0, int T, int cur, void *stream);
int launch_check(const Args &a, int cur, const int *cells, int n_cells, double *out_min_eig,
                 double *out_trace_dev, const void *zref_full, const void *V, void *stream);
// Periodic sweep over every cell (the state of buffers dcur, E of ecur, H of
// hcur): non-finite values set flags[0] bit 0, a population or 2 x 2
// principal minor of the stored state below -tol sets bit 1; in FP32 each
// compensated pair is folded (in FP64) into the canonical pair of its value.
int launch_sweep(const Args &a, int dcur, int ecur, int hcur, double tol, void *stream);
// The same over the owned cells of a batch group's running tiles (tasks of
// the tiled batch, own = cells owned per tile) after the round from step n0.
int launch_sweep_batch(int prec, int N, const Args *args, const int2 *tasks, int n_tasks, int own, long long n0,
                       int cur, double tol, void *stream);
// Smallest density-matrix eigenvalue the state checks accept.
constexpr double EIG_TOL = 1e-6;

// Tensor-core tiled kernel for N = 4..6 (mbs_tc.cu): FP32 state, one medium
// parameter slot, no per-cell operators; tiles of `cells` = 128 or 256 cells
// (one or two 128-row MMA groups per block); T must pass
// tiled_tc_geometry_ok for the grid.
int tiled_tc_supported(int prec, int N);
bool tiled_tc_geometry_ok(int n_cells, int cells, int T);
int launch_tiled_tc(const Args &a, int cells, long long n0, int nsteps, int T, int cur, void *stream);
// Host: the tensor-core tiles' constant table for N levels from the FP64
// parameter block of the medium (layout of q_stride): the TF32 hi/lo weight
// operands in their shared-memory layout, the reference coherences and the
// field angles of the pairs (0, k).  Returns the number of floats written
// (out == nullptr: the number needed).
int tc_weight_table(int N, const double *qblk, float *out);

}  // namespace mbs
