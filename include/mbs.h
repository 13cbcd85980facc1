/*
 * mbs.h -- C ABI of the GB300 Maxwell-Bloch hot path.
 *
 * The library advances the generalized 1D Maxwell-Bloch equations of
 * Riesch & Jirauschek, "mbsolve" (CPC 2021), Sec. 2.1 (Eqs. efield, hfield,
 * master1D and the polarisation term) with the FDTD/operator-splitting
 * scheme of Sec. 2.2 and Algorithm 1 (Sec. 3.2), on one CUDA GPU (sm_103a).
 *
 * Object model (Sec. 3.1): a *device* holds the static setup -- quantum
 * descriptions, materials, regions, cell count, boundary reflectivities --
 * and a *scenario* holds the dynamic part -- Courant number, end time,
 * sources, probes -- plus the device-memory state of one simulation.
 * mbs_solve runs Algorithm 1 for one or more scenarios; mbs_fetch_records
 * copies probe traces to the caller.
 *
 * Conventions (all units SI):
 *   - complex arrays are interleaved (re, im) doubles, matrices row-major;
 *   - the grid has n_cells cells of width dz = length / n_cells; cell m is
 *     centred at (m + 1/2) dz and carries E and rho; H lives on the faces
 *     f = 0..n_cells (face f is the left face of cell f); a cell takes the
 *     material of the first region with x_start <= centre < x_end;
 *   - dt = courant * dz / c_max (c_max the largest light speed among the
 *     cells' materials); n_steps = ceil(t_end / dt) unless given explicitly;
 *   - time step n advances H to n+1/2, rho to n+1/2 (using E^n) and E to n+1;
 *     the density matrix at n = -1/2 is rho_init, E^0 = H^{-1/2} = 0;
 *   - record index n holds E^{n+1} / H^{n+1/2} / rho^{n+1/2}.
 *
 * Ownership: every create call copies its inputs; the caller may free them
 * on return.  Objects are owned by the library until destroyed.  Device
 * memory is allocated by the library (cudaMalloc) on the device current at
 * mbs_scenario time.
 *
 * Errors: every call returns an mbs_status.  On a negative status nothing
 * was created (out pointers are set to NULL) and mbs_last_error() returns a
 * message for the calling thread.  No status is ever reported through a GPU
 * fault: device-side checks set flags that mbs_solve turns into statuses.
 */
#ifndef MBS_H
#define MBS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MBS_ABI_VERSION 2

typedef enum {
    MBS_OK = 0,
    MBS_W_NOT_PSD = 1,     /* warning: the pure-dephasing rates need a
                              non-positive-semidefinite coefficient matrix
                              (Sec. 3.1.1); the object was still created */
    MBS_E_INVALID = -1,    /* invalid argument (see mbs_last_error) */
    MBS_E_CUDA = -2,       /* a CUDA runtime call failed */
    MBS_E_OOM = -3,        /* host or device allocation failed */
    MBS_E_NUMERIC = -4,    /* non-finite state or a density matrix that is
                              not positive semidefinite (beyond tolerance) */
    MBS_E_TIMEOUT = -5,    /* a bounded device-side wait gave up */
    MBS_E_STATE = -6       /* call out of order (e.g. fetch before solve) */
} mbs_status;

typedef struct mbs_device_s *mbs_device_t;
typedef struct mbs_scenario_s *mbs_scenario_t;

/* One quantum-mechanical description (Sec. 3.1.1, class qm_description).
 * Relaxation is the Lindblad dissipator of Eq. (lindbladdiss), given as
 * explicit operators with rates, D(rho) = sum_k g_k (L_k rho L_k^+ -
 * 1/2 {L_k^+ L_k, rho}), and/or in the paper's rate form: the scattering
 * matrix R of Eq. (relax_pop) (R[i*N+j] = gamma_ij, the rate from level j
 * into level i; diagonal ignored) plus the N(N-1)/2 pure-dephasing rates in
 * the order 12, 13, 23, 14, 24, 34, ... .  The rate form is converted to
 * Lindblad operators; if the dephasing rates need a non-PSD coefficient
 * matrix, mbs_device_create returns MBS_W_NOT_PSD and keeps the (then not
 * completely positive) dissipator. */
typedef struct {
    int n_levels;                 /* N >= 2 (tiled FP32 kernels: N = 2, 3) */
    double density;               /* n3D [m^-3], >= 0 */
    const double *h0;             /* N*N complex, Hermitian [J] */
    const double *mu;             /* N*N complex, Hermitian dipole operator [C m] */
    int n_lindblad;               /* >= 0 */
    const double *lindblad_rates; /* [n_lindblad], >= 0 [1/s] */
    const double *lindblad_ops;   /* [n_lindblad][N*N] complex */
    const double *scattering;     /* N*N real or NULL */
    const double *pure_dephasing; /* N(N-1)/2 real or NULL */
    const double *rho_init;       /* N*N complex, Hermitian, trace 1, PSD */
} mbs_qm_desc;

/* Electromagnetic material (Sec. 3.1.1): relative permittivity and
 * permeability, conductivity sigma [S/m], overlap factor Gamma, and the
 * quantum description index (-1: no quantum systems). */
typedef struct { double eps_r, mu_r, sigma, overlap; int qm; } mbs_material;

/* Region [x_start, x_end) [m] made of material `material` (Sec. 3.1.1). */
typedef struct { int material; double x_start, x_end; } mbs_region;

/* Power reflectivity R of the left and right domain ends (Sec. 2.1):
 * 0 = absorbing (first-order Mur), 1 = perfect mirror (E = 0),
 * 0 < R < 1 = partially reflecting facet: with the amplitude reflection
 * r = -sqrt(R) and M the Mur value, the end cell takes
 * E_b^{n+1} = (1 + r) M^{n+1} - r E_b^{n-1} (E_b^{-1} = E_b^0), which at
 * Courant number 1 in vacuum sends back exactly r times the arriving wave.
 * Values outside [0, 1] are rejected with MBS_E_INVALID. */
typedef struct { double refl_left, refl_right; } mbs_bc;

/* Create a device.  per_cell_jitter (optional, NULL = none) holds
 * [n_cells][2] factors (density factor, H0 factor) multiplying n3D and H0
 * of each cell's quantum description.  Validation: Hermitian h0, mu and
 * rho_init (tolerance 1e-12 relative), |tr rho_init - 1| <= 1e-12, rho_init
 * PSD, non-negative rates and density, every cell covered by a region,
 * indices in range, eps_r, mu_r > 0.  Returns MBS_OK, MBS_W_NOT_PSD or an
 * error. */
int mbs_device_create(const mbs_qm_desc *qms, int n_qm,
                      const mbs_material *mats, int n_mat,
                      const mbs_region *regions, int n_regions,
                      double length, int n_cells, mbs_bc bc,
                      const double *per_cell_jitter,
                      mbs_device_t *out);

enum { MBS_SRC_TFSF_RIGHT = 0, /* one-way injection of a +x travelling wave:
                                  total field for m >= cell (needs cell >= 2) */
       MBS_SRC_TFSF_LEFT = 1,  /* one-way -x wave: total field for m <= cell
                                  (needs cell <= n_cells - 3) */
       MBS_SRC_HARD = 2 };     /* E^{n+1} at `cell` is set to the waveform */

enum { MBS_SHAPE_SECH = 0,     /* envelope sech((t - t0)/tau) (class sech_pulse) */
       MBS_SHAPE_GAUSS = 1 };   /* envelope exp(-((t - t0)/tau)^2) (class gaussian_pulse) */

/* Source (Sec. 3.1.2, classes source / sech_pulse / gaussian_pulse):
 * waveform S(t) = e0 envelope(t) sin(omega t + phase) [V/m] with the
 * envelope chosen by `shape`.  Soft sources are total-field/scattered-field
 * injections that add the incident wave and stay transparent to returning
 * waves. */
typedef struct {
    int kind; int cell;
    double e0, tau, t0, omega, phase;
    int shape;                  /* MBS_SHAPE_* */
} mbs_source;

enum { MBS_Q_E = 0,       /* E at the cell centre, E^{n+1} [V/m] */
       MBS_Q_H = 1,       /* H at the left face of the cell, H^{n+1/2} [A/m] */
       MBS_Q_RHO_RE = 2,  /* Re rho_ij^{n+1/2} of the cell */
       MBS_Q_RHO_IM = 3 };/* Im rho_ij^{n+1/2} */

/* Probe (Sec. 3.1.2, class record): one quantity at one cell, recorded
 * every step.  i, j are 0-based level indices for MBS_Q_RHO_*. */
typedef struct { int cell; int quantity; int i, j; } mbs_probe;

/* Create a scenario on `dev`: builds the propagators for dt in FP64 on the
 * host, allocates the device state on the current CUDA device and uploads
 * it.  dt = dt_or_0 if > 0, else courant * dz / c_max (courant in (0, 1]);
 * dt must not exceed dz / c_max.  n_steps > 0 overrides t_end.
 * A two-level medium with per-cell jitter has one set of step operators per
 * cell; those are formed in FP64 on the device (the host's arithmetic, one
 * thread per cell) and only the jitter table is uploaded.  Setting the
 * environment variable MBS_HOST_SETUP to a non-empty value other than "0"
 * when this is called forms them on the host instead (for comparison).  A
 * non-finite per-cell operator returns MBS_E_NUMERIC either way. */
int mbs_scenario(mbs_device_t dev, double dt_or_0, double courant, double t_end, long long n_steps,
                 const mbs_source *src, int n_src,
                 const mbs_probe *probes, int n_probes,
                 mbs_scenario_t *out);

enum { MBS_PREC_FP64 = 0,      /* FP64 state and arithmetic */
       MBS_PREC_FP32 = 1 };    /* FP32 fields and Bloch deviations with
                                  compensated (Kahan) accumulation */
enum { MBS_ALGO_AUTO = 0,
       MBS_ALGO_PLAIN = 1,     /* one thread per cell, two launches per step: H, rho
                                  and d_t P at n + 1/2, then E at n + 1 (the loop
                                  order of Sec. 3.2) */
       MBS_ALGO_TILED = 2 };   /* temporal tiles: tile_steps steps per launch
                                  with halo recompute (the redundant-calculation
                                  loop of Sec. 3.2) */

enum { MBS_SOLVE_ONE_AT_A_TIME = 1,  /* flags: solve batch members one after another */
       MBS_SOLVE_AUTOTUNE = 2,       /* with tile_steps == 0: pick the tile depth by measurement.
                                        Each candidate depth runs one warm-up launch and two
                                        timed rounds of three launches (CUDA events on
                                        cuda_stream) from the current state, which is then
                                        reset; the faster round counts and the fastest per step
                                        wins.  The choice is cached for the process per level
                                        count, precision, kernel variant and cell / step counts
                                        (per batch group: its simulations' totals). */
       MBS_SOLVE_GRAPH = 4 };        /* batched tiled solves on a non-NULL stream: the first call
                                        records the whole launch sequence (fork, every round of
                                        every group, join, state checks) into a CUDA graph and
                                        launches it; later calls with the same scenarios (same
                                        order) and options replay it without rebuilding the task
                                        tables.  Destroying a member scenario frees the graph. */
enum { MBS_SOLVE_TEST_STALL = 1 << 30 };   /* test of the failure path: the tensor-core tiles
                                              (N >= 4) issue no MMA, so every block's bounded
                                              wait on the tensor core expires after about 1 s;
                                              the blocks free their TMEM and return, and
                                              mbs_solve returns MBS_E_TIMEOUT with the CUDA
                                              context intact.  No effect on other kernels. */
enum { MBS_SOLVE_WIDE_TILES = 8 };   /* N >= 4: tensor-core tiles of 256 cells (two 128-row MMA
                                        groups per block) instead of 128; tile_steps must keep the
                                        absorbing ends inside a tile's light cone for the grid
                                        (always true for 1..26) */

typedef struct {
    int precision;     /* MBS_PREC_* */
    int algo;          /* MBS_ALGO_* */
    int tile_steps;    /* steps per tiled launch: N = 2, 3 a multiple of 4 in [4, 32R - 12] (R = 4 cells per
                          lane for N = 2, 2 for N = 3); N >= 4 in [1, 20] (128-cell tiles) or
                          [1, 26] (256-cell tiles; other depths are checked against the grid).
                          0 = the library's choice: measured with MBS_SOLVE_AUTOTUNE (for N >= 4
                          also the tile width), else 32 (N = 2 and 3), 8 / 20 (N >= 4) */
    int check_every;   /* steps between the periodic state checks (Sec. 2.2: the splitting keeps rho a
                          density matrix), 0 = only at the end.  Each check samples the smallest
                          eigenvalue of <= 4096 cells plus the probe cells, and sweeps every cell for
                          non-finite values and for a negative population or 2 x 2 principal minor of
                          the stored state (dipole eigenbasis, tolerance 1e-6); in FP32 the sweep
                          also folds each compensated (Kahan) pair into the canonical pair of its
                          value, in FP64.  A failed check makes every later step launch of the
                          scenario return at once.  A single scenario's solve reads the status at
                          each check and stops there (MBS_E_NUMERIC, the step count in
                          mbs_scenario_stats); a batch reads it when all members have finished, the
                          failing member having stopped at its check (tile rounds are the
                          boundaries: a check runs after the round that crosses a multiple of
                          check_every).  Records of the steps after a failed check are not written. */
    int flags;         /* MBS_SOLVE_* */
} mbs_opts;

/* Run every scenario from its initial condition to its last step (previous
 * results are discarded).  `cuda_stream` is a cudaStream_t or NULL for the
 * legacy default stream.  The call returns after the work has completed.
 * Several scenarios on the tiled path (algo AUTO or TILED, no
 * MBS_SOLVE_ONE_AT_A_TIME) advance together, grouped by kernel variant (level
 * count and parameter layout): each round of a group's tile_steps steps is
 * one launch over the blocks of the group's scenarios still running
 * (scenarios may differ in cells, steps and parameters).  With more than one
 * group, each group runs on a stream forked from cuda_stream and joined back
 * into it.
 * Returns MBS_E_NUMERIC if a state check found a non-finite value or a
 * density-matrix eigenvalue below -1e-6 (in a batch: the first such status,
 * after every member has finished). */
int mbs_solve(mbs_scenario_t *batch, int n_scen, const mbs_opts *opts, void *cuda_stream);

/* Copy probe `probe`'s trace (n_steps doubles, SI units) into out.  With
 * out == NULL only *n_written is set (the required count).  Returns
 * MBS_E_INVALID if cap is too small, MBS_E_STATE before the first solve. */
int mbs_fetch_records(mbs_scenario_t s, int probe, double *out, size_t cap, size_t *n_written);

/* Initial field E^0 of the scenario (Sec. 2.1 initial conditions), one
 * value per cell [V/m], copied; e0 == NULL restores the default zero field.
 * H^{-1/2} stays zero.  Used by every later solve.  n must equal n_cells;
 * non-finite values are rejected. */
int mbs_scenario_set_field(mbs_scenario_t s, const double *e0, size_t n);

/* Grid facts of a scenario: dt [s], dz [m], number of steps. */
int mbs_scenario_info(mbs_scenario_t s, double *dt, double *dz, long long *n_steps);

/* State diagnostics of the last solve over the probe cells and a strided
 * sample of medium cells (FP64 on the device): max |tr rho - 1|, smallest
 * eigenvalue of rho, number of steps run. */
int mbs_scenario_stats(mbs_scenario_t s, double *max_trace_dev, double *min_eig, long long *n_steps);

/* Host-side introspection of the FP64 setup (no GPU needed): for quantum
 * description `qm` of `dev` at time step dt, the real generator in the
 * dipole eigenbasis and the derived step operators.  With N levels,
 * K = N*N - 1 and P = N(N-1)/2, each non-NULL output receives:
 *   lambda[N]     eigenvalues of mu (ascending) [C m]
 *   V[N*N]        complex eigenvectors of mu (columns), interleaved
 *   A[K*K]        linear part of one full step exp(L0 dt) on Bloch
 *                 deviations (row-major)
 *   Ah[N*N*N*N]   exp(L0 dt/2) on the full real coordinates
 *   c[K]          affine offset of exp(L0 dt) at the reference state
 *   zref[N*N]     reference state (full real coordinates)
 *   g[K], g0      d_t P / n3D = g . u + g0 for the rotated deviation u
 * The real coordinates of rho are, in the eigenbasis of mu (rho~ = V^+ rho
 * V): rho~_kk for k < N, then Re rho~_jk, Im rho~_jk for the pairs j < k in
 * the order (0,1), (0,2), ..., (0,N-1), (1,2), ... ; the Bloch deviation
 * coordinates drop rho~_{N-1,N-1}. */
int mbs_device_propagators(mbs_device_t dev, int qm, double dt,
                           double *lambda, double *V, double *A, double *Ah,
                           double *c, double *zref, double *g, double *g0);

/* Tile depth (steps per tiled launch) the last solve used, 0 for the plain
 * path; MBS_E_STATE before the first solve. */
int mbs_scenario_tile(mbs_scenario_t s, int *tile_steps);

/* The tile plan of the tiled kernels (the temporal tiles with redundant
 * halo computation of Sec. 3.2), a pure host query (no device work):
 * whether `tile_steps` steps per launch are valid for tiles of `tile_cells`
 * cells on an `nx`-cell grid with `n_levels` levels, and how many tiles one
 * launch runs.  tile_cells = 512 for N = 2 and 3 (tile_steps a multiple of
 * 4 in [4, 116] for N = 2, [4, 52] for N = 3, any nx); 128 or 256 for the
 * tensor-core tiles of N = 4..6 (the tile that holds the last cell starts 4
 * or 8 cells early when that cell would be its first owned cell or start a
 * warp; tile_steps is valid when the last cell and its neighbour then stay
 * owned, in one warp and inside the light cone, and so do cell 0 and its
 * neighbour).  Tile b owns cells [b own, (b + 1) own), own = tile_cells -
 * 2 tile_steps.  MBS_OK with *n_tiles set, or MBS_E_INVALID. */
int mbs_tile_plan(int n_levels, int tile_cells, int nx, int tile_steps, int *n_tiles);

/* Cells per tile of the last solve's tiled launches (Sec. 3.2; each tile owns
 * tile_cells - 2 tile_steps of them): 512 for N = 2 and 3, 128 or 256 for
 * the tensor-core tiles of N >= 4 (the autotuner may pick either); 0 for the
 * plain path; MBS_E_STATE before the first solve. */
int mbs_scenario_tile_cells(mbs_scenario_t s, int *tile_cells);

/* Transfer and launch counters: bytes copied host -> device by the
 * scenario's creation and its solves so far, bytes copied device -> host by
 * the last solve and the fetches after it, CUDA kernel launches issued by
 * the last solve. */
int mbs_scenario_counters(mbs_scenario_t s, long long *h2d_bytes, long long *d2h_bytes,
                          long long *kernel_launches);

/* Largest number of density matrices mbs_check_rho_static accepts per call. */
#define MBS_STATIC_CHECK_MAX 65536

/* Density-matrix check that allocates no device memory.  It has no
 * counterpart in the paper: it exists for callers that cannot call
 * cudaMalloc -- a framework that owns every device allocation through its
 * own pool, or a loop that must not stall on the device-wide
 * synchronisation an allocation can imply -- and still want the
 * positivity/trace check that mbs_solve applies to its own state.
 *   rho       device pointer, n matrices of n_levels x n_levels complex
 *             (interleaved re, im, row-major), read only
 *   n         1 .. MBS_STATIC_CHECK_MAX (larger n: MBS_E_INVALID, no work)
 *   n_levels  2 .. 6
 *   out       device pointer to 3 doubles, written: smallest eigenvalue of
 *             the Hermitian parts of the finite matrices (NaN when no matrix
 *             is finite), largest |tr rho - 1| over the finite matrices (0
 *             when there is none), number of matrices with a non-finite
 *             entry
 *   cuda_stream  cudaStream_t or NULL; the call only enqueues work on it
 *             (asynchronous with respect to the host).
 * Scratch: a fixed static device array of 3 doubles per matrix for
 * MBS_STATIC_CHECK_MAX matrices (1.5 MB), held by every GPU that loads the
 * library until the process exits.  No cudaMalloc, cudaFree or other
 * allocating call is made.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current and caches
 * it for the process; make that first call before any stream capture, and
 * do not call the entry point on a device after cudaDeviceReset (the cached
 * address does not survive it).  Every call shares the array and it keeps
 * the last call's contents; each call writes the n entries it then reads, so
 * nothing needs clearing, but calls that overlap on the GPU (on different
 * streams, or from several host threads) race on it. */
int mbs_check_rho_static(const double *rho, int n, int n_levels, double *out, void *cuda_stream);

/* Arithmetic peak of the current GPU, measured by a small kernel, for the
 * rooflines of the kernels above (the paper has no counterpart).
 *   which  0: FP32 fused multiply-add (8 independent chains per thread, 8
 *             blocks of 256 threads per SM); the FP32 lanes also set the
 *             instruction-issue limit, one warp instruction per scheduler and
 *             clock, so rate / 64 is the issue peak in warp instructions/s;
 *          1: FP64 fused multiply-add (the same shape);
 *          2: TF32 tensor-core MMA, tcgen05.mma kind::tf32 with M = 128,
 *             N = 256, K = 8 from shared memory into TMEM, issued back to back
 *             by one thread of one block per SM (every wait bounded: a wait
 *             that gives up returns MBS_E_TIMEOUT).
 *   rate     out: flop/s of the last of three launches (the first two warm up)
 *   seconds  out (or NULL): that launch's duration
 *   cuda_stream  cudaStream_t or NULL; the call synchronises on its events.
 * Allocates and frees a small device buffer. */
int mbs_peak_rates(int which, double *rate, double *seconds, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Driven single cells (Sec. 2.1, the borderline case Nx = 1: with one grid
 * point the method integrates the Lindblad master equation alone; the
 * V-type three-level application example of Sec. 4 is one such system).  A batch of
 * n_sys independent systems, each with its own quantum description and its
 * own prescribed field
 *   E^n = e0 envelope(t_n) sin(omega t_n + phase),  t_n = n dt
 *   (the source's shape: sech((t - t0)/tau) or exp(-((t - t0)/tau)^2)),
 *   E^0 = 0 (the initial field),
 * advances n_steps steps of the Strang splitting of Sec. 2.2 (step n uses
 * E^n, as a grid cell under a hard source does).  One GPU thread per system.
 * The populations rho_kk^{n+1/2} are recorded every record_every steps:
 * record r holds step n = (r + 1) record_every - 1.  The density n3D and the
 * source kind are not used (no field is fed back). */
typedef struct mbs_cells_s *mbs_cells_t;

/* Build the batch on the host (FP64 step operators per system; systems with
 * the same tau, t0, omega, phase share one tabulated drive shape).  All
 * systems must have the same level count, 2 or 3.  Inputs are copied.
 * Returns MBS_OK, MBS_W_NOT_PSD (some system's dephasing rates) or an error
 * (MBS_E_INVALID with the offending system in mbs_last_error). */
int mbs_cells_create(const mbs_qm_desc *qms, int n_sys, double dt, long long n_steps,
                     const mbs_source *drives, int record_every, mbs_cells_t *out);

/* Run all systems from their initial states (FP32 with compensated sums, or
 * FP64) on `cuda_stream` (cudaStream_t or NULL); device memory is allocated
 * on the current device on the first solve of each precision.  Returns
 * after completion; MBS_E_NUMERIC if a final density matrix is not finite or
 * has an eigenvalue below -1e-6. */
int mbs_cells_solve(mbs_cells_t c, int precision, void *cuda_stream);

/* Copy system `sys`'s records, n_rec x N doubles (out[r N + k] =
 * rho_kk of record r), n_rec = n_steps / record_every.  out == NULL: only
 * *n_written (the count) is set. */
int mbs_cells_fetch(mbs_cells_t c, int sys, double *out, size_t cap, size_t *n_written);

/* Over all systems after the last solve: max |tr rho - 1|, smallest
 * eigenvalue of rho. */
int mbs_cells_stats(mbs_cells_t c, double *max_trace_dev, double *min_eig);

void mbs_cells_destroy(mbs_cells_t c);

void mbs_scenario_destroy(mbs_scenario_t s);
void mbs_device_destroy(mbs_device_t d);

/* Message for the last non-OK status on the calling thread ("" if none). */
const char *mbs_last_error(void);

/* Library version, equals MBS_ABI_VERSION. */
int mbs_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MBS_H */
