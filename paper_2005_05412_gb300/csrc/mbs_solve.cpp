// mbs_solve.cpp -- the solve of one scenario (the loop of Sec. 3.2, plain
// or in temporal tiles with redundant halo calculations), the periodic
// state checks (Sec. 2.2: the splitting keeps rho a density matrix), the
// tile-depth autotuner, and mbs_solve, which sends batches of several
// scenarios to mbs_batch.cpp.
#include <algorithm>
#include <array>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "mbs_host_internal.h"

namespace mbs_host {

int prepare_solve(mbs_scenario_s *s, int prec, cudaStream_t st) {
  g_h2d = &s->h2d_bytes;
  int rc = ensure_bundle(s, prec);
  g_h2d = nullptr;
  if (rc) return rc;
  s->d2h_bytes = 0;
  s->launches = 0;
  Bundle &b = s->b[prec];
  const size_t row = (size_t)s->ld * b.rb;
  const int K = s->K;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    if ((e = cudaMemsetAsync(b.E[i], 0, row, st)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(b.H[i], 0, row, st)) != cudaSuccess) break;
    if (b.El[i] && (e = cudaMemsetAsync(b.El[i], 0, row, st)) != cudaSuccess) break;
    if (b.Hl[i] && (e = cudaMemsetAsync(b.Hl[i], 0, row, st)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(b.C[i], 0, row * K, st)) != cudaSuccess) break;
    e = cudaMemcpyAsync(b.D[i], b.Dinit, row * K, cudaMemcpyDeviceToDevice, st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b.pd, 0, row, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_flags, 0, 4 * sizeof(int), st);
  // the initial field E^0 (also E^{-1}: a static field before the first step)
  double eb[2] = {0.0, 0.0};
  if (e == cudaSuccess && !s->e_init.empty()) {
    const int nx = s->dev->nx;
    eb[0] = s->e_init[0];
    eb[1] = s->e_init[nx - 1];
    if (prec == 0) {
      for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync((double *)b.E[i] + s->off, s->e_init.data(), nx * sizeof(double), cudaMemcpyHostToDevice, st);
    } else {
      s->e_init_f.resize(2 * (size_t)nx);
      for (int m = 0; m < nx; ++m) {
        const float hi = (float)s->e_init[m];
        s->e_init_f[m] = hi;
        s->e_init_f[nx + m] = (float)(s->e_init[m] - (double)hi);
      }
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMemcpyAsync((float *)b.E[i] + s->off, s->e_init_f.data(), nx * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync((float *)b.El[i] + s->off, s->e_init_f.data() + nx, nx * sizeof(float),
                              cudaMemcpyHostToDevice, st);
      }
    }
  }
  if (e == cudaSuccess) {
    if (prec == 0) {
      s->bprev_init_d = {eb[0], 0.0, eb[1], 0.0};
      for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(b.bprev[i], s->bprev_init_d.data(), 4 * sizeof(double), cudaMemcpyHostToDevice, st);
    } else {
      const float l = (float)eb[0], r = (float)eb[1];
      s->bprev_init_f = {l, (float)(eb[0] - (double)l), r, (float)(eb[1] - (double)r)};
      for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaMemcpyAsync(b.bprev[i], s->bprev_init_f.data(), 4 * sizeof(float), cudaMemcpyHostToDevice, st);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "state reset");
  return MBS_OK;
}

// Tile depth when the caller leaves it to the library: the fastest measured
// on GB300 (two and three levels: 32 steps, tensor-core tiles: 8 for
// 128 cells, 20 for 256 cells).
int default_tile_steps(int N, int tc_cells) { return N <= 3 ? 32 : tc_cells == 256 ? 20 : 8; }

// Whether scenario s runs on the tensor-core tiles (N = 4..6 in FP32 with a
// single medium and no per-cell operators).
bool uses_tc(const mbs_scenario_s *s, int prec) {
  return s->N >= 4 && mbs::tiled_tc_supported(prec, s->N) && s->n_slot == 1 && !s->has_pcell;
}

int default_algo(const mbs_scenario_s *s, int prec) {
  if (uses_tc(s, prec)) return MBS_ALGO_TILED;
  return mbs::tiled_supported(prec, s->N) && (!s->has_pcell || s->N == 2) ? MBS_ALGO_TILED : MBS_ALGO_PLAIN;
}

// Whether the tiled kernels cover scenario s with tile depth T (sets the error).
int tiled_ok(const mbs_scenario_s *s, int prec, int T) {
  if (s->N >= 4) {
    if (!uses_tc(s, prec))
      return fail(MBS_E_INVALID,
                  "tiled kernels for N >= 4 need FP32, one medium and no per-cell factors; use the plain algorithm");
    if (!mbs::tiled_tc_geometry_ok(s->dev->nx, s->tc_cells, T))
      return fail(MBS_E_INVALID,
                  "tile_steps %d does not fit %d-cell tensor-core tiles on this grid (1..20 always fit 128-cell tiles)",
                  T, s->tc_cells);
    return MBS_OK;
  }
  if (!mbs::tiled_supported(prec, s->N) || (s->has_pcell && s->N != 2))
    return fail(MBS_E_INVALID, "tiled kernels cover N = 2 (also with per-cell factors) and N = 3");
  const int R = mbs::tile_lane_cells(s->N);
  if (T % 4 != 0 || T < 4 || T > mbs::tile_max_steps(s->N))
    return fail(MBS_E_INVALID, "tile_steps must be a multiple of 4 in [4, %d]", mbs::tile_max_steps(s->N) / 4 * 4);
  // each lane's R-cell group must hold at most one medium material
  for (int g = 0; g * R < s->dev->nx; ++g) {
    int sl = -1;
    for (int j = 0; j < R && g * R + j < s->dev->nx; ++j) {
      const int q = s->qslot[s->dev->cell_mat[g * R + j]];
      if (q >= 0 && sl >= 0 && q != sl)
        return fail(MBS_E_INVALID, "two media meet inside a %d-cell group; use the plain algorithm", R);
      if (q >= 0) sl = q;
    }
  }
  return MBS_OK;
}

int launch_state_check(mbs_scenario_s *s, const mbs::Args &a, int c, cudaStream_t st) {
  const int nchk = (int)s->chk_cells.size();
  if (!nchk) return 0;
  ++s->launches;
  return mbs::launch_check(a, c, s->d_chk_cells, nchk, s->d_chk_min, s->d_chk_tr, s->d_zref, nullptr, st);
}

// The periodic check of Sec. 2.2's density-matrix properties at a step
// boundary: the sampled eigenvalue check, then the sweep over every cell
// (finiteness, populations and 2 x 2 minors; the FP32 Kahan fold).  With
// `wait` the host reads the status at once and returns true if it failed,
// so that the caller stops issuing launches; either way a failed check makes
// every later step launch of the scenario return at once.
int periodic_check(mbs_scenario_s *s, const mbs::Args &a, int dcur, int ecur, int hcur, cudaStream_t st,
                          bool wait, bool *failed) {
  int r = launch_state_check(s, a, dcur, st);
  if (!r) {
    ++s->launches;
    r = mbs::launch_sweep(a, dcur, ecur, hcur, mbs::EIG_TOL, st);
  }
  if (r) return cuda_fail((cudaError_t)r, "check launch");
  *failed = false;
  if (wait) {
    int flags[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(flags, s->d_flags, sizeof flags, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "check status");
    s->d2h_bytes += sizeof flags;
    *failed = flags[0] != 0 || flags[1] != 0;
  }
  return MBS_OK;
}

// After the stream has drained: read the check results and device flags.
int finish_solve(mbs_scenario_s *s, int prec, int cur, long long steps_run) {
  cudaError_t e;
  s->solved_prec = prec;
  s->last_cur = cur;
  s->steps_run = steps_run < 0 ? s->nt : steps_run;
  const int nchk = (int)s->chk_cells.size();
  int flags[4] = {0, 0, 0, 0};
  if ((e = cudaMemcpy(flags, s->d_flags, sizeof flags, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "flags");
  s->d2h_bytes += sizeof flags + (long long)nchk * 2 * sizeof(double);
  s->st_min = 1e300;
  s->st_trace = 0;
  if (nchk) {
    std::vector<double> mn(nchk), tr(nchk);
    if ((e = cudaMemcpy(mn.data(), s->d_chk_min, nchk * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(tr.data(), s->d_chk_tr, nchk * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "check results");
    for (int i = 0; i < nchk; ++i) {
      s->st_min = std::min(s->st_min, mn[i]);
      s->st_trace = std::max(s->st_trace, tr[i]);
    }
  } else {
    s->st_min = 0;
  }
  if (flags[1]) return fail(MBS_E_TIMEOUT, "a bounded wait on the tensor cores gave up");
  if (flags[0] & 1) return fail(MBS_E_NUMERIC, "non-finite state after %lld steps", s->steps_run);
  if (flags[0]) return fail(MBS_E_NUMERIC, "density matrix not positive semidefinite after %lld steps", s->steps_run);
  if (nchk && s->st_min < -1e-6) return fail(MBS_E_NUMERIC, "density matrix eigenvalue %.3g < -1e-6", s->st_min);
  return MBS_OK;
}

// ------------------------------------------------------------ autotuning
// Tile depth by measurement: every candidate depth runs one warm-up launch and
// two timed rounds of three launches (CUDA events on the solve stream) of the
// scenario (or of the whole batch group) from its current state; the faster
// round counts and the fastest time per step wins.  The caller resets the state afterwards.  Results are cached for the
// process, keyed by level count, precision, kernel variant and the cell and
// step counts, so a workload shape is tuned once.
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;

std::vector<int> tile_candidates(int N, long long nt) {
  std::vector<int> c = N >= 4 ? std::vector<int>{6, 8, 10, 12, 14, 16, 20}
                     : N == 3 ? std::vector<int>{16, 20, 24, 28, 32, 40, 48}
                              : std::vector<int>{12, 16, 20, 24, 28, 32, 40, 48};
  std::vector<int> out;
  for (int T : c)
    if (T <= nt) out.push_back(T);
  return out;
}

static int tiled_launch(const mbs_scenario_s *s, const mbs::Args &a, long long n0, int ns, int T, int cur,
                        cudaStream_t st) {
  return s->N >= 4 ? mbs::launch_tiled_tc(a, s->tc_cells, n0, ns, T, cur, st)
                   : mbs::launch_tiled(a, n0, ns, T, cur, st);
}


// returns the winning candidate code (see code_steps / code_cells)
static int autotune_one(mbs_scenario_s *s, int prec, const mbs::Args &a, cudaStream_t st) {
  char key[128];
  std::snprintf(key, sizeof key, "1:%d:%d:%d:%d:%d", s->N, prec, s->N >= 4 ? 9 : mbs::tiled_variant(a), s->dev->nx,
                (int)std::min<long long>(s->nt, 1 << 30));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
  }
  std::vector<int> cands;
  for (int T : tile_candidates(s->N, s->nt)) {
    if (s->N < 4) {
      if (T <= mbs::tile_max_steps(s->N)) cands.push_back(T);
      continue;
    }
    if (mbs::tiled_tc_geometry_ok(s->dev->nx, 128, T)) cands.push_back(T);
  }
  if (s->N >= 4)
    for (int T : {12, 16, 20, 24, 32, 40})
      if (T <= s->nt && mbs::tiled_tc_geometry_ok(s->dev->nx, 256, T)) cands.push_back(1000 + T);
  if (cands.size() < 2) return default_tile_steps(s->N);
  const int saved = s->tc_cells;
  const int T = tune_loop(cands, st, [&](int c, int cur) {
    s->tc_cells = code_cells(c);
    return tiled_launch(s, a, 0, code_steps(c), code_steps(c), cur, st);
  });
  s->tc_cells = saved;
  if (T < 0) return default_tile_steps(s->N);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = T;
  return T;
}

int solve_one(mbs_scenario_s *s, const mbs_opts &o, cudaStream_t st) {
  const int prec = o.precision;
  int rc = prepare_solve(s, prec, st);
  if (rc) return rc;
  mbs::Args a = make_args(s, prec);
  int algo = o.algo == MBS_ALGO_AUTO ? default_algo(s, prec) : o.algo;
  s->tc_cells = (o.flags & MBS_SOLVE_WIDE_TILES) ? 256 : 128;
  a.test_stall = (o.flags & MBS_SOLVE_TEST_STALL) ? 1 : 0;
  int T = o.tile_steps > 0 ? o.tile_steps : default_tile_steps(s->N, s->tc_cells);
  const int chk = o.check_every > 0 ? o.check_every : 0;
  int cur = 0;
  long long done = 0;
  bool stopped = false;   // a periodic check failed
  if (algo == MBS_ALGO_TILED) {
    if ((rc = tiled_ok(s, prec, T))) return rc;
    if (o.tile_steps <= 0 && (o.flags & MBS_SOLVE_AUTOTUNE)) {
      const int code = autotune_one(s, prec, a, st);
      T = code_steps(code);
      if (s->N >= 4) s->tc_cells = code_cells(code);
      if ((rc = prepare_solve(s, prec, st))) return rc;   // the trials advanced the state
    }
    while (done < s->nt && !stopped) {
      const int ns = (int)std::min<long long>(T, s->nt - done);
      int r = tiled_launch(s, a, done, ns, T, cur, st);
      ++s->launches;
      if (r) return cuda_fail((cudaError_t)r, "tiled launch");
      cur ^= 1;
      done += ns;
      if (chk && done < s->nt && (done / chk) != ((done - ns) / chk))
        if ((r = periodic_check(s, a, cur, cur, cur, st, true, &stopped))) return r;
    }
    s->tile_used = T;
  } else {
    for (long long n = 0; n < s->nt && !stopped; ++n) {
      int r = mbs::launch_plain_step(a, n, cur, st);
      s->launches += 2;
      if (r) return cuda_fail((cudaError_t)r, "plain launch");
      cur ^= 1;
      done = n + 1;
      if (chk && (n + 1) % chk == 0 && n + 1 < s->nt)   // plain: D, H in buffers 0, E in cur
        if ((r = periodic_check(s, a, 0, cur, 0, st, true, &stopped))) return r;
    }
    s->tile_used = 0;
  }
  // plain: D, H live in buffer 0, E in `cur`; tiled: everything in `cur`
  const int dcur = algo == MBS_ALGO_TILED ? cur : 0;
  if ((rc = launch_state_check(s, a, dcur, st))) return cuda_fail((cudaError_t)rc, "check launch");
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "solve");
  return finish_solve(s, prec, cur, done);
}

}  // namespace mbs_host

using namespace mbs_host;

extern "C" {

int mbs_solve(mbs_scenario_t *batch, int n_scen, const mbs_opts *opts, void *cuda_stream) {
  g_err.clear();
  if (!batch || n_scen < 1) return fail(MBS_E_INVALID, "empty batch");
  mbs_opts o{MBS_PREC_FP32, MBS_ALGO_AUTO, 0, 0, 0};
  if (opts) o = *opts;
  if (o.precision != MBS_PREC_FP64 && o.precision != MBS_PREC_FP32) return fail(MBS_E_INVALID, "bad precision");
  if (o.algo < 0 || o.algo > 2) return fail(MBS_E_INVALID, "bad algorithm");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  for (int i = 0; i < n_scen; ++i)
    if (!batch[i]) return fail(MBS_E_INVALID, "scenario %d is NULL", i);
  // several scenarios on the tiled path advance together, unless asked not to
  bool batched = n_scen > 1 && !(o.flags & MBS_SOLVE_ONE_AT_A_TIME) && o.algo != MBS_ALGO_PLAIN;
  for (int i = 0; i < n_scen && batched; ++i)
    batched = batch[i]->N <= 3 && default_algo(batch[i], o.precision) == MBS_ALGO_TILED;
  if (batched) {
    std::vector<mbs_scenario_s *> ss(batch, batch + n_scen);
    return solve_batch(ss, o, st);
  }
  for (int i = 0; i < n_scen; ++i) {
    const int rc = solve_one(batch[i], o, st);
    if (rc) return rc;
  }
  return MBS_OK;
}

}  // extern "C"
