// mbs_batch.cpp -- batched solves: many independent simulations advance
// together, one launch per round of tile_steps steps over the blocks of the
// simulations still running, grouped by kernel variant, optionally recorded
// once as a CUDA graph and replayed.
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

// Batched tiled solve: every round launches, per kernel variant, one grid
// over the blocks of all simulations still running, advancing them T steps.
// Blocks are ordered by their simulation's step count (longest first), so
// the running ones form a prefix and the grid shrinks as simulations end.
struct BatchGroup {
  int N, pm, T;
  std::vector<int> sims;   // indices into the batch, longest first
  std::vector<int2> tasks;
  std::vector<long long> task_nt;
  int max_mat = 0, max_slot = 0, max_stride = 0;
};

void group_tasks(BatchGroup &g, const std::vector<mbs_scenario_s *> &ss, int T,
                        std::vector<int2> &tasks, std::vector<long long> &task_nt) {
  tasks.clear();
  task_nt.clear();
  const int own = mbs::tile_own(g.N, T);
  for (int i : g.sims) {
    const int n_tiles = (ss[i]->dev->nx + own - 1) / own;
    for (int w = 0; w < n_tiles; ++w) {
      tasks.push_back(make_int2(i, w));
      task_nt.push_back(ss[i]->nt);
    }
  }
}

// A batched solve recorded as a CUDA graph (MBS_SOLVE_GRAPH), with the device
// tables its launches read; replayed while the same scenarios are solved with
// the same options.  Destroying a member scenario drops the graph.
struct BatchGraph {
  std::vector<mbs_scenario_s *> members;
  int prec = 0, tile = 0, flags = 0, check_every = 0;
  std::vector<int> Ts;      // tile depth per group
  std::vector<int> sim_T;   // tile depth per member
  cudaGraphExec_t exec = nullptr;
  mbs::Args *d_args = nullptr;
  std::vector<int2 *> d_tasks;
};
static std::mutex g_graph_mu;
static std::vector<BatchGraph *> g_graphs;

void free_graph(BatchGraph *g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  cudaFree(g->d_args);
  for (auto *p : g->d_tasks) cudaFree(p);
  delete g;
}

void drop_graphs_of(mbs_scenario_s *s) {
  std::lock_guard<std::mutex> lk(g_graph_mu);
  for (size_t k = 0; k < g_graphs.size();) {
    auto &m = g_graphs[k]->members;
    if (std::find(m.begin(), m.end(), s) != m.end()) {
      free_graph(g_graphs[k]);
      g_graphs.erase(g_graphs.begin() + k);
    } else {
      ++k;
    }
  }
}

int solve_batch(std::vector<mbs_scenario_s *> &ss, const mbs_opts &o, cudaStream_t st) {
  const int prec = o.precision;
  const int chk = o.check_every > 0 ? o.check_every : 0;
  int rc;
  for (auto *s : ss) {
    if ((rc = prepare_solve(s, prec, st))) return rc;
    if ((rc = tiled_ok(s, prec, o.tile_steps > 0 ? o.tile_steps : default_tile_steps(s->N)))) return rc;
  }
  // graphs need a stream that can be captured (not the legacy default stream)
  const bool use_graph = (o.flags & MBS_SOLVE_GRAPH) != 0 && st != nullptr;
  // replay a recorded graph of this very batch
  if (use_graph) {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    for (auto *g : g_graphs)
      if (g->members == ss && g->prec == prec && g->tile == o.tile_steps && g->flags == o.flags &&
          g->check_every == chk) {
        cudaError_t e = cudaGraphLaunch(g->exec, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "batched graph replay");
        int status = MBS_OK;
        for (size_t i = 0; i < ss.size(); ++i) {
          const int T = g->sim_T[i];
          const long long rounds = (ss[i]->nt + T - 1) / T;
          ss[i]->launches = rounds;
          ss[i]->tile_used = T;
          rc = finish_solve(ss[i], prec, (int)(rounds % 2));
          if (rc && status == MBS_OK) status = rc;
        }
        return status;
      }
  }
  std::vector<BatchGroup> groups;
  std::vector<mbs::Args> args(ss.size());
  for (size_t i = 0; i < ss.size(); ++i) {
    args[i] = make_args(ss[i], prec);
    const int pm = mbs::tiled_variant(args[i]);
    if (pm < 0) return fail(MBS_E_INVALID, "scenario %zu is not covered by the tiled kernels", i);
    BatchGroup *g = nullptr;
    for (auto &x : groups)
      if (x.N == ss[i]->N && x.pm == pm) g = &x;
    if (!g) {
      groups.push_back(BatchGroup{ss[i]->N, pm, o.tile_steps > 0 ? o.tile_steps : default_tile_steps(ss[i]->N)});
      g = &groups.back();
    }
    g->sims.push_back((int)i);
    g->max_mat = std::max(g->max_mat, args[i].n_mat_all);
    g->max_slot = std::max(g->max_slot, args[i].n_slot);
    g->max_stride = std::max(g->max_stride, args[i].qstride);
  }
  for (auto &g : groups)
    std::stable_sort(g.sims.begin(), g.sims.end(), [&](int x, int y) { return ss[x]->nt > ss[y]->nt; });
  // device copy of the per-simulation arguments
  mbs::Args *d_args = nullptr;
  std::vector<int2 *> d_tasks(groups.size(), nullptr);
  auto cleanup = [&]() {
    cudaFree(d_args);
    for (auto *p : d_tasks) cudaFree(p);
  };
  cudaError_t e = cudaMalloc(&d_args, args.size() * sizeof(mbs::Args));
  if (e == cudaSuccess) e = cudaMemcpy(d_args, args.data(), args.size() * sizeof(mbs::Args), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "batch tables");
  }
  // tile depth per group: given, default, or measured
  if (o.tile_steps <= 0 && (o.flags & MBS_SOLVE_AUTOTUNE)) {
    for (auto &g : groups) {
      long long nt_min = LLONG_MAX, cells = 0, steps = 0;
      for (int i : g.sims) {
        nt_min = std::min(nt_min, ss[i]->nt);
        cells += ss[i]->dev->nx;
        steps += ss[i]->nt;
      }
      char key[160];
      std::snprintf(key, sizeof key, "B:%d:%d:%d:%zu:%lld:%lld", g.N, prec, g.pm, g.sims.size(), cells, steps);
      int T = -1;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) T = it->second;
      }
      if (T < 0) {
        std::vector<int> cands;
        for (int t : tile_candidates(g.N, nt_min))
          if (t <= mbs::tile_max_steps(g.N)) cands.push_back(t);
        const size_t smem = mbs::tiled_batch_smem(prec, g.N, g.max_mat, g.max_slot, g.max_stride);
        std::vector<int2> tk;
        std::vector<long long> tn;
        int2 *d_tk = nullptr;
        int last_T = -1;
        T = tune_loop(cands, st, [&](int t, int cur) {
          if (t != last_T) {   // tasks of this depth
            if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
            cudaFree(d_tk);
            d_tk = nullptr;
            group_tasks(g, ss, t, tk, tn);
            if (cudaMalloc(&d_tk, tk.size() * sizeof(int2)) != cudaSuccess ||
                cudaMemcpy(d_tk, tk.data(), tk.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
              return -1;
            last_T = t;
          }
          return mbs::launch_tiled_batch(prec, g.N, g.pm, d_args, d_tk, (int)tk.size(), smem, 0, t, cur, st);
        });
        cudaStreamSynchronize(st);
        cudaFree(d_tk);
        if (T < 0) T = default_tile_steps(g.N);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[key] = T;
      }
      g.T = T;
    }
    for (auto *s : ss)   // the trials advanced the state
      if ((rc = prepare_solve(s, prec, st))) {
        cleanup();
        return rc;
      }
  }
  for (size_t k = 0; k < groups.size() && e == cudaSuccess; ++k) {
    group_tasks(groups[k], ss, groups[k].T, groups[k].tasks, groups[k].task_nt);
    e = cudaMalloc(&d_tasks[k], groups[k].tasks.size() * sizeof(int2));
    if (e == cudaSuccess)
      e = cudaMemcpy(d_tasks[k], groups[k].tasks.data(), groups[k].tasks.size() * sizeof(int2),
                     cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "batch tables");
  }
  std::vector<int> sim_T(ss.size());
  for (const auto &g : groups)
    for (int i : g.sims) sim_T[i] = g.T;
  // Each group runs on a stream of its own, forked from and joined back into
  // the caller's stream, so that one group's last, thinly populated rounds
  // overlap the other group's work.
  const size_t n_fork = groups.size() > 1 ? groups.size() : 0;
  std::vector<cudaStream_t> gst(groups.size(), st);
  std::vector<cudaEvent_t> ev(n_fork + 1, nullptr);
  auto release = [&]() {
    for (size_t k = 0; k < n_fork; ++k)
      if (gst[k] != st) cudaStreamDestroy(gst[k]);
    for (auto x : ev)
      if (x) cudaEventDestroy(x);
  };
  for (size_t k = 0; k < n_fork && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&gst[k], cudaStreamNonBlocking);
    if (e != cudaSuccess) gst[k] = st;
  }
  for (size_t k = 0; k < ev.size() && n_fork && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    release();
    cleanup();
    return cuda_fail(e, "batch streams");
  }
  // the launch sequence: fork, every group's rounds, join, per-simulation checks
  auto enqueue = [&]() -> int {
    cudaError_t x = cudaSuccess;
    if (n_fork) x = cudaEventRecord(ev[n_fork], st);
    for (size_t k = 0; k < n_fork && x == cudaSuccess; ++k) x = cudaStreamWaitEvent(gst[k], ev[n_fork], 0);
    if (x != cudaSuccess) return cuda_fail(x, "batch streams");
    for (size_t k = 0; k < groups.size(); ++k) {
      const auto &g = groups[k];
      const size_t smem = mbs::tiled_batch_smem(prec, g.N, g.max_mat, g.max_slot, g.max_stride);
      const long long nt_max = g.task_nt.front();
      int cur = 0;
      for (long long n0 = 0; n0 < nt_max; n0 += g.T) {
        // running blocks: a prefix of the tasks (sorted by step count)
        const int active = (int)(std::upper_bound(g.task_nt.begin(), g.task_nt.end(), n0,
                                                  [](long long v, long long y) { return v > y; }) -
                                 g.task_nt.begin());
        int r = mbs::launch_tiled_batch(prec, g.N, g.pm, d_args, d_tasks[k], active, smem, n0, g.T, cur, gst[k]);
        if (r) return cuda_fail((cudaError_t)r, "batched tiled launch");
        cur ^= 1;
        // periodic check: the sweep over every cell of the simulations that
        // ran this round (a failure stops that simulation's later rounds on
        // the device; the status is read when the batch has finished)
        const long long n1 = n0 + g.T;
        if (chk && n1 < nt_max && n1 / chk != n0 / chk) {
          r = mbs::launch_sweep_batch(prec, g.N, d_args, d_tasks[k], active, mbs::tile_own(g.N, g.T), n0, cur,
                                      mbs::EIG_TOL, gst[k]);
          if (r) return cuda_fail((cudaError_t)r, "batched sweep launch");
        }
      }
    }
    for (size_t k = 0; k < n_fork && x == cudaSuccess; ++k) {
      x = cudaEventRecord(ev[k], gst[k]);
      if (x == cudaSuccess) x = cudaStreamWaitEvent(st, ev[k], 0);
    }
    if (x != cudaSuccess) return cuda_fail(x, "batch streams");
    for (size_t i = 0; i < ss.size(); ++i) {
      const long long rounds = (ss[i]->nt + sim_T[i] - 1) / sim_T[i];
      const int r = launch_state_check(ss[i], args[i], (int)(rounds % 2), st);
      if (r) return cuda_fail((cudaError_t)r, "check launch");
    }
    return MBS_OK;
  };
  BatchGraph *graph = nullptr;
  if (use_graph) {
    cudaGraph_t gr = nullptr;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      release();
      cleanup();
      return cuda_fail(e, "graph capture (a NULL or legacy stream cannot be captured)");
    }
    rc = enqueue();
    const cudaError_t e2 = cudaStreamEndCapture(st, &gr);
    if (rc == MBS_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "graph capture");
    graph = new BatchGraph;
    if (rc == MBS_OK && (e = cudaGraphInstantiate(&graph->exec, gr, 0)) != cudaSuccess)
      rc = cuda_fail(e, "graph instantiation");
    if (gr) cudaGraphDestroy(gr);
    if (rc == MBS_OK && (e = cudaGraphLaunch(graph->exec, st)) != cudaSuccess) rc = cuda_fail(e, "graph launch");
    if (rc != MBS_OK) {
      free_graph(graph);
      release();
      cleanup();
      return rc;
    }
  } else {
    rc = enqueue();
    if (rc != MBS_OK) {
      cudaStreamSynchronize(st);
      release();
      cleanup();
      return rc;
    }
  }
  e = cudaStreamSynchronize(st);
  release();
  if (graph) {   // the graph keeps the tables it reads
    graph->members = ss;
    graph->prec = prec;
    graph->tile = o.tile_steps;
    graph->flags = o.flags;
    graph->check_every = chk;
    for (const auto &g : groups) graph->Ts.push_back(g.T);
    graph->sim_T = sim_T;
    graph->d_args = d_args;
    graph->d_tasks = d_tasks;
    std::lock_guard<std::mutex> lk(g_graph_mu);
    g_graphs.push_back(graph);
  } else {
    cleanup();
  }
  if (e != cudaSuccess) return cuda_fail(e, "batched solve");
  int status = MBS_OK;
  for (size_t i = 0; i < ss.size(); ++i) {
    auto *s = ss[i];
    const long long rounds = (s->nt + sim_T[i] - 1) / sim_T[i];
    s->launches = rounds;
    s->tile_used = sim_T[i];
    rc = finish_solve(s, prec, (int)(rounds % 2));
    if (rc && status == MBS_OK) status = rc;
  }
  return status;
}

}  // namespace mbs_host
