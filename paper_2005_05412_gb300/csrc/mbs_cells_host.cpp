// mbs_cells_host.cpp -- host side of the driven single cells (Sec. 2.1,
// the borderline case Nx = 1): setup, device tables, solve and fetch of a
// batch of independent driven systems (kernels in mbs_cells.cu).
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

using namespace mbs_host;

// ============================================================ driven cells
// Batched single-cell Lindblad solver (include/mbs.h, mbs_cells_*): Nx = 1,
// the master equation of each system under its prescribed field.
struct mbs_cells_s {
  int N = 0, K = 0, P = 0, n_sys = 0, every = 1, rows = 0, n_tab = 0;
  double dt = 0;
  long long nt = 0, n_rec = 0;
  std::vector<double> prm, amp, tab, zref, Dinit;   // FP64 master copies
  std::vector<int> tab_id;
  struct Dev {
    bool ready = false;
    void *prm = nullptr, *D = nullptr, *C = nullptr, *amp = nullptr, *tab = nullptr, *rec = nullptr;
  } b[2];
  int *d_tab_id = nullptr, *d_flags = nullptr;
  double *d_zref = nullptr, *d_min = nullptr, *d_tr = nullptr;
  int solved_prec = -1;
  double st_min = 0, st_trace = 0;
};

namespace {
using namespace mbs_host;

void free_cells(mbs_cells_s *c) {
  for (auto &b : c->b) {
    cudaFree(b.prm);
    cudaFree(b.D);
    cudaFree(b.C);
    cudaFree(b.amp);
    cudaFree(b.tab);
    cudaFree(b.rec);
    b = mbs_cells_s::Dev();
  }
  cudaFree(c->d_tab_id);
  cudaFree(c->d_flags);
  cudaFree(c->d_zref);
  cudaFree(c->d_min);
  cudaFree(c->d_tr);
}

int cells_device(mbs_cells_s *c, int prec) {
  auto &b = c->b[prec];
  if (!b.ready) {
    const size_t rb = rsize(prec), ns = (size_t)c->n_sys;
    int rc;
    if ((rc = upload(c->prm, &b.prm, prec)) || (rc = upload(c->amp, &b.amp, prec))) return rc;
    cudaError_t e = cudaMalloc(&b.D, ns * c->K * rb);
    if (e == cudaSuccess) e = cudaMalloc(&b.C, ns * c->K * rb);
    if (e == cudaSuccess) e = cudaMalloc(&b.rec, std::max<size_t>(1, (size_t)c->n_rec * c->N * ns) * rb);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (cells)");
    if (prec == 0) {
      if ((rc = upload(c->tab, &b.tab, 0))) return rc;
    } else {   // [n_tab][2][nt]: high words, then low words of each shape
      std::vector<float> f(2 * c->tab.size());
      for (int t = 0; t < c->n_tab; ++t)
        for (long long n = 0; n < c->nt; ++n) {
          const double v = c->tab[(size_t)t * c->nt + n];
          const float hi = (float)v;
          f[(size_t)t * 2 * c->nt + n] = hi;
          f[(size_t)t * 2 * c->nt + c->nt + n] = (float)(v - (double)hi);
        }
      if ((e = cudaMalloc(&b.tab, f.size() * sizeof(float))) != cudaSuccess ||
          (e = cudaMemcpy(b.tab, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "drive tables");
    }
    b.ready = true;
  }
  if (!c->d_flags) {
    int rc;
    if ((rc = upload_raw(c->tab_id, &c->d_tab_id)) || (rc = upload_raw(c->zref, &c->d_zref))) return rc;
    cudaError_t e = cudaMalloc(&c->d_flags, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_min, c->n_sys * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_tr, c->n_sys * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (cells)");
  }
  return MBS_OK;
}

}  // namespace

extern "C" {

int mbs_cells_create(const mbs_qm_desc *qms, int n_sys, double dt, long long n_steps, const mbs_source *drives,
                     int record_every, mbs_cells_t *out) {
  g_err.clear();
  if (!out) return fail(MBS_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!qms || !drives || n_sys < 1) return fail(MBS_E_INVALID, "need n_sys >= 1 systems and their drives");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(MBS_E_INVALID, "dt must be > 0");
  if (n_steps < 1 || n_steps > (1LL << 31)) return fail(MBS_E_INVALID, "n_steps must be in [1, 2^31]");
  if (record_every < 1) return fail(MBS_E_INVALID, "record_every must be >= 1");
  const int N = qms[0].n_levels;
  if (N != 2 && N != 3) return fail(MBS_E_INVALID, "driven cells: n_levels must be 2 or 3");
  auto c = std::make_unique<mbs_cells_s>();
  c->N = N;
  c->K = N * N - 1;
  c->P = N * (N - 1) / 2;
  c->n_sys = n_sys;
  c->dt = dt;
  c->nt = n_steps;
  c->every = record_every;
  c->n_rec = n_steps / record_every;
  const int K = c->K, P = c->P, N2 = N * N;
  c->rows = K * K + K + 3 * P + N * (K + 1);
  c->prm.assign((size_t)c->rows * n_sys, 0.0);
  c->zref.assign((size_t)n_sys * N2, 0.0);
  c->Dinit.assign((size_t)K * n_sys, 0.0);
  c->amp.assign(n_sys, 0.0);
  c->tab_id.assign(n_sys, 0);
  int status = MBS_OK;
  // drive shapes: systems with the same (tau, t0, omega, phase) share one
  std::vector<std::array<double, 5>> shapes;
  for (int s = 0; s < n_sys; ++s) {
    const mbs_source &d = drives[s];
    if (!std::isfinite(d.e0) || !std::isfinite(d.tau) || !std::isfinite(d.t0) || !std::isfinite(d.omega) ||
        !std::isfinite(d.phase) || !(d.tau > 0))
      return fail(MBS_E_INVALID, "system %d: drive parameters must be finite with tau > 0", s);
    if (d.shape != MBS_SHAPE_SECH && d.shape != MBS_SHAPE_GAUSS) return fail(MBS_E_INVALID, "system %d: bad shape", s);
    const std::array<double, 5> k{d.tau, d.t0, d.omega, d.phase, (double)d.shape};
    int id = -1;
    for (size_t j = 0; j < shapes.size() && id < 0; ++j)
      if (shapes[j] == k) id = (int)j;
    if (id < 0) {
      id = (int)shapes.size();
      shapes.push_back(k);
    }
    c->tab_id[s] = id;
    c->amp[s] = d.e0;
  }
  c->n_tab = (int)shapes.size();
  // E^n = e0 envelope((t_n - t0)/tau) sin(omega t_n + phase), t_n = n dt; E^0 = 0
  c->tab.assign((size_t)c->n_tab * n_steps, 0.0);
  for (int j = 0; j < c->n_tab; ++j)
    for (long long n = 1; n < n_steps; ++n) {
      const double t = (double)n * dt;
      c->tab[(size_t)j * n_steps + n] =
          std::sin(shapes[j][2] * t + shapes[j][3]) * envelope((int)shapes[j][4], (t - shapes[j][1]) / shapes[j][0]);
    }
  std::vector<int> codes(n_sys, MBS_OK);
  std::vector<std::string> msgs(n_sys);
#pragma omp parallel for schedule(dynamic, 16)
  for (int s = 0; s < n_sys; ++s) {
    if (qms[s].n_levels != N) {
      codes[s] = MBS_E_INVALID;
      msgs[s] = "all systems must have the same number of levels";
      continue;
    }
    QDesc q;
    const int rc = build_qdesc(qms[s], q);
    if (rc < 0) {
      codes[s] = rc;
      msgs[s] = g_err;
      continue;
    }
    codes[s] = rc;
    Step st;
    build_step(q, 1.0, dt, st);
    auto put = [&](int row, double v) { c->prm[(size_t)row * n_sys + s] = v; };
    for (int i = 0; i < K * K; ++i) put(i, st.AKm1[i]);
    for (int i = 0; i < K; ++i) put(K * K + i, st.c[i]);
    int p = 0;
    for (int j = 0; j < N; ++j)
      for (int k = j + 1; k < N; ++k, ++p) {
        put(K * K + K + p, (q.lambda[j] - q.lambda[k]) * dt / kHbar);
        put(K * K + K + P + 2 * p, q.yref[N + 2 * p]);
        put(K * K + K + P + 2 * p + 1, q.yref[N + 2 * p + 1]);
      }
    for (int k = 0; k < N; ++k) {   // rho_kk^{n+1/2} = coef . u + coef_K
      const std::vector<double> h = rho_functional(q, k, k, false);
      std::vector<double> hA(N2, 0.0);
      for (int cc = 0; cc < N2; ++cc)
        for (int r = 0; r < N2; ++r) hA[cc] += h[r] * st.Ah[r * N2 + cc];
      double h0 = 0;
      for (int cc = 0; cc < N2; ++cc) h0 += hA[cc] * q.yref[cc];
      const int r0 = K * K + K + 3 * P + k * (K + 1);
      for (int i = 0; i < K; ++i) put(r0 + i, hA[full_of(N, i)] - (i < N - 1 ? hA[N - 1] : 0.0));
      put(r0 + K, h0);
    }
    std::vector<double> x0(N2, 0.0);
    for (int i = 0; i < N2; ++i)
      for (int j = 0; j < N2; ++j) x0[i] += st.Ehm1[i * N2 + j] * q.yinit[j];
    for (int i = 0; i < K; ++i)
      c->Dinit[(size_t)i * n_sys + s] = x0[full_of(N, i)] + (q.yinit[full_of(N, i)] - q.yref[full_of(N, i)]);
    std::copy(q.yref.begin(), q.yref.end(), &c->zref[(size_t)s * N2]);
  }
  for (int s = 0; s < n_sys; ++s) {
    if (codes[s] < 0) return fail(codes[s], "system %d: %s", s, msgs[s].c_str());
    if (codes[s] == MBS_W_NOT_PSD) status = MBS_W_NOT_PSD;
  }
  for (double v : c->prm)
    if (!std::isfinite(v)) return fail(MBS_E_NUMERIC, "non-finite step operator (check H0, mu, rates and dt)");
  *out = c.release();
  return status;
}

int mbs_cells_solve(mbs_cells_t c, int precision, void *cuda_stream) {
  g_err.clear();
  if (!c) return fail(MBS_E_INVALID, "cells is NULL");
  if (precision != MBS_PREC_FP64 && precision != MBS_PREC_FP32) return fail(MBS_E_INVALID, "bad precision");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int rc = cells_device(c, precision);
  if (rc) return rc;
  auto &b = c->b[precision];
  const size_t rb = rsize(precision), ns = (size_t)c->n_sys;
  cudaError_t e;
  if (precision == 0) {
    e = cudaMemcpyAsync(b.D, c->Dinit.data(), c->Dinit.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  } else {
    std::vector<float> f(c->Dinit.begin(), c->Dinit.end());
    e = cudaMemcpyAsync(b.D, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // f leaves scope
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(b.C, 0, ns * c->K * rb, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_flags, 0, 4 * sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "cells state reset");
  mbs::CellsArgs a{};
  a.prec = precision;
  a.N = c->N;
  a.n_sys = c->n_sys;
  a.nt = c->nt;
  a.every = c->every;
  a.prm = b.prm;
  a.D = b.D;
  a.C = b.C;
  a.amp = b.amp;
  a.tab_id = c->d_tab_id;
  a.tab = b.tab;
  a.tab_stride = precision == 0 ? c->nt : 2 * c->nt;
  a.rec = b.rec;
  a.zref = c->d_zref;
  a.flags = c->d_flags;
  constexpr long long CHUNK = 2048;   // steps per launch
  for (long long n0 = 0; n0 < c->nt; n0 += CHUNK) {
    const int ns_ = (int)std::min<long long>(CHUNK, c->nt - n0);
    if ((rc = mbs::launch_cells(a, n0, ns_, st))) return cuda_fail((cudaError_t)rc, "cells launch");
  }
  if ((rc = mbs::launch_cells_check(a, c->d_min, c->d_tr, st))) return cuda_fail((cudaError_t)rc, "cells check");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cells solve");
  int flags[4];
  std::vector<double> mn(c->n_sys), tr(c->n_sys);
  if ((e = cudaMemcpy(flags, c->d_flags, sizeof flags, cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(mn.data(), c->d_min, ns * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
      (e = cudaMemcpy(tr.data(), c->d_tr, ns * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cells check results");
  c->solved_prec = precision;
  c->st_min = *std::min_element(mn.begin(), mn.end());
  c->st_trace = *std::max_element(tr.begin(), tr.end());
  if (flags[0]) return fail(MBS_E_NUMERIC, "non-finite density matrix");
  if (c->st_min < -1e-6) return fail(MBS_E_NUMERIC, "density matrix eigenvalue %.3g < -1e-6", c->st_min);
  return MBS_OK;
}

int mbs_cells_fetch(mbs_cells_t c, int sys, double *out, size_t cap, size_t *n_written) {
  g_err.clear();
  if (!c) return fail(MBS_E_INVALID, "cells is NULL");
  if (sys < 0 || sys >= c->n_sys) return fail(MBS_E_INVALID, "system index out of range");
  const size_t n = (size_t)c->n_rec * c->N;
  if (n_written) *n_written = n;
  if (!out) return MBS_OK;
  if (cap < n) return fail(MBS_E_INVALID, "capacity %zu < %zu", cap, n);
  if (c->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  if (n == 0) return MBS_OK;
  const size_t rb = rsize(c->solved_prec);
  // element (r, k) of system sys sits at (r N + k) n_sys + sys
  const char *src = static_cast<const char *>(c->b[c->solved_prec].rec) + (size_t)sys * rb;
  cudaError_t e;
  if (c->solved_prec == 0) {
    e = cudaMemcpy2D(out, rb, src, (size_t)c->n_sys * rb, rb, n, cudaMemcpyDeviceToHost);
  } else {
    std::vector<float> f(n);
    e = cudaMemcpy2D(f.data(), rb, src, (size_t)c->n_sys * rb, rb, n, cudaMemcpyDeviceToHost);
    for (size_t i = 0; i < n; ++i) out[i] = f[i];
  }
  if (e != cudaSuccess) return cuda_fail(e, "cells fetch");
  return MBS_OK;
}

int mbs_cells_stats(mbs_cells_t c, double *max_trace_dev, double *min_eig) {
  g_err.clear();
  if (!c) return fail(MBS_E_INVALID, "cells is NULL");
  if (c->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  if (max_trace_dev) *max_trace_dev = c->st_trace;
  if (min_eig) *min_eig = c->st_min;
  return MBS_OK;
}

void mbs_cells_destroy(mbs_cells_t c) {
  if (!c) return;
  free_cells(c);
  delete c;
}

}  // extern "C"
