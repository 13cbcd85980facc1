// mbs_host.cpp -- host side of the GB300 Maxwell-Bloch hot path: the
// objects of the C ABI (include/mbs.h) -- device (static setup: quantum
// descriptions, materials, regions, reflectivities) and scenario (time
// step, sources, probes and the device-memory state of one simulation) --
// with their validation, tables and device buffers, and the query calls.
// The FP64 step operators come from mbs_setup.cpp, the solves from
// mbs_solve.cpp and mbs_batch.cpp.
#include <algorithm>
#include <array>
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "mbs_host_internal.h"
#include "mbs_setup_dev.h"
#include "mbs_step_math.h"

namespace mbs_host {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? MBS_E_OOM : MBS_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

thread_local long long *g_h2d = nullptr;

size_t rsize(int prec) { return prec == 0 ? sizeof(double) : sizeof(float); }


// upload a double vector as `prec` reals
int upload(const std::vector<double> &h, void **dptr, int prec) {
  const size_t n = h.size();
  if (n == 0) {
    *dptr = nullptr;
    return 0;
  }
  cudaError_t e = cudaMalloc(dptr, n * rsize(prec));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  if (g_h2d) *g_h2d += (long long)(n * rsize(prec));
  if (prec == 0) {
    e = cudaMemcpy(*dptr, h.data(), n * sizeof(double), cudaMemcpyHostToDevice);
  } else {
    std::vector<float> f(n);
#pragma omp parallel for schedule(static) if (n > 65536)
    for (size_t i = 0; i < n; ++i) f[i] = (float)h[i];
    e = cudaMemcpy(*dptr, f.data(), n * sizeof(float), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  return 0;
}

// per-step source table: FP64 as is; FP32 as [2][nt] high and low words of
// each value (v = hi + lo to ~2^-48 relative)
int upload_src(const std::vector<double> &h, void **dptr, int prec) {
  if (prec == 0) return upload(h, dptr, 0);
  const size_t n = h.size();
  std::vector<float> f(2 * n);
  for (size_t i = 0; i < n; ++i) {
    f[i] = (float)h[i];
    f[n + i] = (float)(h[i] - (double)f[i]);
  }
  cudaError_t e = cudaMalloc(dptr, f.size() * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  if (g_h2d) *g_h2d += (long long)(f.size() * sizeof(float));
  e = cudaMemcpy(*dptr, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  return 0;
}


void free_bundle(Bundle &b) {
  for (int i = 0; i < 2; ++i) {
    cudaFree(b.E[i]);
    cudaFree(b.H[i]);
    cudaFree(b.El[i]);
    cudaFree(b.Hl[i]);
    cudaFree(b.D[i]);
    cudaFree(b.C[i]);
  }
  cudaFree(b.pd);
  cudaFree(b.Dinit);
  cudaFree(b.emc);
  cudaFree(b.qpar);
  cudaFree(b.pcell);
  cudaFree(b.pcell2);
  cudaFree(b.pr_coef);
  cudaFree(b.rec);
  cudaFree(b.tcw);
  cudaFree(b.bprev[0]);
  cudaFree(b.bprev[1]);
  for (void *p : b.src_tabs) cudaFree(p);
  b = Bundle();
}

int ensure_bundle(mbs_scenario_s *s, int prec) {
  Bundle &b = s->b[prec];
  if (b.ready) return 0;
  const size_t rb = rsize(prec);
  b.rb = rb;
  const size_t row = (size_t)s->ld * rb;
  const int K = s->K;
  cudaError_t e;
  for (int i = 0; i < 2; ++i) {
    if ((e = cudaMalloc(&b.E[i], row)) != cudaSuccess) return cuda_fail(e, "cudaMalloc E");
    if ((e = cudaMalloc(&b.H[i], row)) != cudaSuccess) return cuda_fail(e, "cudaMalloc H");
    if (prec == 1) {
      if ((e = cudaMalloc(&b.El[i], row)) != cudaSuccess) return cuda_fail(e, "cudaMalloc El");
      if ((e = cudaMalloc(&b.Hl[i], row)) != cudaSuccess) return cuda_fail(e, "cudaMalloc Hl");
    }
    if ((e = cudaMalloc(&b.D[i], row * std::max(K, 1))) != cudaSuccess) return cuda_fail(e, "cudaMalloc D");
    if ((e = cudaMalloc(&b.C[i], row * std::max(K, 1))) != cudaSuccess) return cuda_fail(e, "cudaMalloc C");
  }
  if ((e = cudaMalloc(&b.pd, row)) != cudaSuccess) return cuda_fail(e, "cudaMalloc pd");
  for (int i = 0; i < 2; ++i)
    if ((e = cudaMalloc(&b.bprev[i], 4 * rb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc bprev");
  int rc;
  // rows formed on the device (jittered two-level media) in `prec`: a copy
  // (FP64) or a conversion (FP32) of the scenario's FP64 rows
  auto from_dev = [&](const double *src, size_t n, void **dst) -> int {
    cudaError_t e2 = cudaMalloc(dst, n * rb);
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaMalloc");
    if (prec == 0) {
      e2 = cudaMemcpy(*dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice);
      if (e2 != cudaSuccess) return cuda_fail(e2, "cudaMemcpy");
    } else {
      const int r2 = mbs::to_float(src, reinterpret_cast<float *>(*dst), n, nullptr);
      if (r2) return cuda_fail((cudaError_t)r2, "FP32 copy of the per-cell rows");
      if ((e2 = cudaStreamSynchronize(nullptr)) != cudaSuccess) return cuda_fail(e2, "FP32 copy of the per-cell rows");
    }
    return 0;
  };
  if (s->d_dinit64) {
    if ((rc = from_dev(s->d_dinit64, (size_t)K * s->ld, &b.Dinit))) return rc;
    if ((rc = from_dev(s->d_pcell64, (size_t)mbs::pc_rows(s->N) * s->ld, &b.pcell))) return rc;
    if (s->has_b2 && (rc = from_dev(s->d_pcell2_64, (size_t)7 * s->ld, &b.pcell2))) return rc;
  } else {
    if ((rc = upload(s->Dinit, &b.Dinit, prec))) return rc;
    if (s->has_pcell && (rc = upload(s->pcell, &b.pcell, prec))) return rc;
    if (s->has_b2 && (rc = upload(s->pcell2, &b.pcell2, prec))) return rc;
  }
  if ((rc = upload(s->emc, &b.emc, prec))) return rc;
  if ((rc = upload(s->qpar, &b.qpar, prec))) return rc;
  if (prec == 1) {
    // FP32 records of rho probes hold rho_ab - rho_ab(ref) (the constant term
    // is added in FP64 when the records are fetched), so that a population
    // near 1 keeps the full FP32 precision of its deviation
    std::vector<double> co = s->pr_coef;
    const int K = s->K;
    for (size_t k = 0; k < s->pr_cell.size(); ++k) co[k * (K + 1) + K] = 0.0;
    if ((rc = upload(co, &b.pr_coef, prec))) return rc;
  } else if ((rc = upload(s->pr_coef, &b.pr_coef, prec))) {
    return rc;
  }
  if (prec == 1 && !s->tcw.empty() && (rc = upload_raw(s->tcw, &b.tcw))) return rc;
  const size_t nrec = std::max<size_t>(1, s->pr_cell.size()) * (size_t)s->nt;
  if ((e = cudaMalloc(&b.rec, nrec * rb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc records");
  if ((e = cudaMemset(b.rec, 0, nrec * rb)) != cudaSuccess) return cuda_fail(e, "cudaMemset");
  for (auto &sr : s->src) {
    void *p = nullptr;
    if ((rc = upload_src(sr.sH, &p, prec))) return rc;
    b.src_tabs.push_back(p);
    if ((rc = upload_src(sr.sE, &p, prec))) return rc;
    b.src_tabs.push_back(p);
  }
  b.ready = true;
  return 0;
}

mbs::Args make_args(mbs_scenario_s *s, int prec) {
  Bundle &b = s->b[prec];
  mbs::Args a{};
  a.prec = prec;
  a.N = s->N;
  a.K = s->K;
  a.P = s->P;
  a.nx = s->dev->nx;
  a.ld = s->ld;
  a.off = s->off;
  a.nt = s->nt;
  for (int i = 0; i < 2; ++i) {
    a.E[i] = b.E[i];
    a.H[i] = b.H[i];
    a.El[i] = b.El[i];
    a.Hl[i] = b.Hl[i];
    a.D[i] = b.D[i];
    a.C[i] = b.C[i];
  }
  a.pd = b.pd;
  a.mat = s->d_mat;
  a.n_mat_all = (int)s->qslot.size();
  a.emc = b.emc;
  a.qslot = s->d_qslot;
  a.qpar = b.qpar;
  a.n_slot = s->n_slot;
  a.qstride = s->qstride;
  a.pcell = s->has_pcell ? b.pcell : nullptr;
  a.pcell2 = s->has_b2 ? b.pcell2 : nullptr;

  a.n_src = (int)s->src.size();
  for (size_t k = 0; k < s->src.size(); ++k) {
    a.src[k].kind = s->src[k].kind;
    a.src[k].face = s->src[k].face;
    a.src[k].cell = s->src[k].cell;
    a.src[k].sH = b.src_tabs[2 * k];
    a.src[k].sE = b.src_tabs[2 * k + 1];
  }
  a.bc_l = s->dev->bc_l;
  a.bc_r = s->dev->bc_r;
  a.r_l = s->dev->r_l;
  a.r_r = s->dev->r_r;
  a.bprev[0] = b.bprev[0];
  a.bprev[1] = b.bprev[1];
  a.kmur_l = s->kmur_l;
  a.kmur_r = s->kmur_r;
  a.n_probe = (int)s->pr_cell.size();
  a.pr_cell = s->d_pr_cell;
  a.pr_q = s->d_pr_q;
  a.pr_coef = b.pr_coef;
  a.tcw = b.tcw;
  a.rec = b.rec;
  a.zref = s->d_zref;
  a.flags = s->d_flags;
  return a;
}

void free_scenario(mbs_scenario_s *s) {
  for (auto &b : s->b) free_bundle(b);
  cudaFree(s->d_mat);
  cudaFree(s->d_qslot);
  cudaFree(s->d_pr_cell);
  cudaFree(s->d_pr_q);
  cudaFree(s->d_flags);
  cudaFree(s->d_chk_cells);
  cudaFree(s->d_zref);
  cudaFree(s->d_chk_min);
  cudaFree(s->d_chk_tr);
  cudaFree(s->d_pcell64);
  cudaFree(s->d_pcell2_64);
  cudaFree(s->d_dinit64);
}

double light_speed(const MatDesc &m) { return 1.0 / std::sqrt(kEps0 * m.eps_r * kMu0 * m.mu_r); }

// source envelopes (Sec. 3.1.2, sech_pulse / gaussian_pulse) at x = (t - t0)/tau
double envelope(int shape, double x) { return shape == MBS_SHAPE_GAUSS ? std::exp(-x * x) : 1.0 / std::cosh(x); }

}  // namespace mbs_host

using namespace mbs_host;

int mbs::set_error(int code, const char *msg) { return fail(code, "%s", msg); }

// ============================================================ C ABI
extern "C" {

const char *mbs_last_error(void) { return g_err.c_str(); }

int mbs_abi_version(void) { return MBS_ABI_VERSION; }

int mbs_device_create(const mbs_qm_desc *qms, int n_qm, const mbs_material *mats, int n_mat,
                      const mbs_region *regions, int n_regions, double length, int n_cells, mbs_bc bc,
                      const double *per_cell_jitter, mbs_device_t *out) {
  g_err.clear();
  if (!out) return fail(MBS_E_INVALID, "out is NULL");
  *out = nullptr;
  if (n_qm < 0 || (n_qm > 0 && !qms)) return fail(MBS_E_INVALID, "bad quantum description list");
  if (n_mat < 1 || n_mat > 250 || !mats) return fail(MBS_E_INVALID, "need 1..250 materials");
  if (n_regions < 1 || !regions) return fail(MBS_E_INVALID, "need at least one region");
  if (!(length > 0) || n_cells < 8) return fail(MBS_E_INVALID, "need length > 0 and n_cells >= 8");
  if (n_cells > (1 << 30)) return fail(MBS_E_INVALID, "n_cells too large");
  // 0: absorbing (first-order Mur), 1: mirror, 2: partially reflecting
  auto refl = [](double r) { return r == 0.0 ? 0 : (r == 1.0 ? 1 : (r > 0.0 && r < 1.0 ? 2 : -1)); };
  if (refl(bc.refl_left) < 0 || refl(bc.refl_right) < 0)
    return fail(MBS_E_INVALID, "reflectivity must be in [0, 1]");
  auto dev = std::make_unique<mbs_device_s>();
  dev->nx = n_cells;
  dev->length = length;
  dev->dz = length / n_cells;
  dev->bc_l = refl(bc.refl_left);
  dev->bc_r = refl(bc.refl_right);
  dev->r_l = -std::sqrt(bc.refl_left);
  dev->r_r = -std::sqrt(bc.refl_right);
  int status = MBS_OK;
  for (int i = 0; i < n_qm; ++i) {
    QDesc q;
    const int rc = build_qdesc(qms[i], q);
    if (rc < 0) return rc;
    if (rc == MBS_W_NOT_PSD) status = MBS_W_NOT_PSD;
    dev->qms.push_back(std::move(q));
  }
  for (int i = 0; i < n_mat; ++i) {
    const mbs_material &m = mats[i];
    if (!(m.eps_r > 0) || !(m.mu_r > 0) || !(m.sigma >= 0) || !(m.overlap >= 0))
      return fail(MBS_E_INVALID, "material %d: need eps_r, mu_r > 0, sigma, overlap >= 0", i);
    if (m.qm < -1 || m.qm >= n_qm) return fail(MBS_E_INVALID, "material %d: bad quantum description index", i);
    dev->mats.push_back({m.eps_r, m.mu_r, m.sigma, m.overlap, m.qm});
  }
  for (int r = 0; r < n_regions; ++r)
    if (regions[r].material < 0 || regions[r].material >= n_mat)
      return fail(MBS_E_INVALID, "region %d: bad material index", r);
  dev->cell_mat.resize(n_cells);
  for (int m = 0; m < n_cells; ++m) {
    const double x = (m + 0.5) * dev->dz;
    int k = -1;
    for (int r = 0; r < n_regions; ++r)
      if (x >= regions[r].x_start && x < regions[r].x_end) {
        k = regions[r].material;
        break;
      }
    if (k < 0) return fail(MBS_E_INVALID, "cell %d (x = %g m) lies in no region", m, x);
    dev->cell_mat[m] = (uint8_t)k;
    const int q = dev->mats[k].qm;
    if (q >= 0) {
      if (dev->N == 0) dev->N = dev->qms[q].N;
      if (dev->qms[q].N != dev->N) return fail(MBS_E_INVALID, "media with different level counts in one device");
    }
  }
  if (per_cell_jitter) {
    dev->jitter.assign(per_cell_jitter, per_cell_jitter + (size_t)2 * n_cells);
    for (double v : dev->jitter)
      if (!std::isfinite(v) || v < 0) return fail(MBS_E_INVALID, "per-cell factors must be finite and >= 0");
  }
  *out = dev.release();
  return status;
}

void mbs_device_destroy(mbs_device_t d) { delete d; }

int mbs_device_propagators(mbs_device_t dev, int qm, double dt, double *lambda, double *V, double *A,
                           double *Ah, double *c, double *zref, double *g, double *g0) {
  g_err.clear();
  if (!dev || qm < 0 || qm >= (int)dev->qms.size() || !(dt > 0)) return fail(MBS_E_INVALID, "bad arguments");
  const QDesc &q = dev->qms[qm];
  const int N = q.N, N2 = N * N, K = N2 - 1;
  Step s;
  build_step(q, 1.0, dt, s);
  if (lambda) std::copy(q.lambda.begin(), q.lambda.end(), lambda);
  if (V)
    for (int i = 0; i < N2; ++i) {
      V[2 * i] = q.V[i].real();
      V[2 * i + 1] = q.V[i].imag();
    }
  if (A) std::copy(s.AK.begin(), s.AK.end(), A);
  if (Ah) std::copy(s.Ah.begin(), s.Ah.end(), Ah);
  if (c) std::copy(s.c.begin(), s.c.end(), c);
  if (zref) std::copy(q.yref.begin(), q.yref.end(), zref);
  if (g) std::copy(s.g.begin(), s.g.end(), g);
  if (g0) *g0 = s.g0;
  (void)K;
  return MBS_OK;
}

// The per-cell operators of a jittered two-level medium on the device
// (mbs_setup_dev.cu): the per-slot FP64 parts and the jitter table go up,
// the FP64 rows stay on the device (the bundles copy or convert them), and
// the two counts come back: a non-finite operator fails the scenario, a cell
// without the optical-Bloch pattern turns the structured rows off.
static int setup_on_device(mbs_scenario_s *s, const std::vector<int> &slot_mat, double dt) {
  const mbs_device_s *dev = s->dev;
  const int nx = dev->nx, ld = s->ld, K = s->K;
  std::vector<mbs::SetupSlot2> slots(s->n_slot);
  for (int sl = 0; sl < s->n_slot; ++sl) {
    const MatDesc &mm = dev->mats[slot_mat[sl]];
    const QDesc &q = dev->qms[mm.qm];
    mbs::SetupSlot2 &o = slots[sl];
    std::copy(q.MH.begin(), q.MH.end(), o.MH);
    std::copy(q.MD.begin(), q.MD.end(), o.MD);
    std::copy(q.yref.begin(), q.yref.end(), o.yref);
    std::copy(q.yinit.begin(), q.yinit.end(), o.yinit);
    std::copy(q.lambda.begin(), q.lambda.end(), o.lambda);
    const double bp = (dt / (kEps0 * mm.eps_r)) / (1 + dt * mm.sigma / (2 * kEps0 * mm.eps_r));
    o.cpl0 = bp * mm.overlap * q.n3d;
  }
  mbs::SetupSlot2 *d_slots = nullptr;
  double *d_jit = nullptr;
  int *d_counts = nullptr;
  int rc = 0;
  g_h2d = &s->h2d_bytes;
  rc = upload_raw(slots, &d_slots);
  if (!rc) rc = upload_raw(dev->jitter, &d_jit);
  g_h2d = nullptr;
  cudaError_t e = cudaSuccess;
  const size_t pr = (size_t)mbs::pc_rows(s->N) * ld, p2 = (size_t)7 * ld, di = (size_t)K * ld;
  if (!rc && ((e = cudaMalloc(&s->d_pcell64, pr * sizeof(double))) != cudaSuccess ||
              (e = cudaMalloc(&s->d_pcell2_64, p2 * sizeof(double))) != cudaSuccess ||
              (e = cudaMalloc(&s->d_dinit64, di * sizeof(double))) != cudaSuccess ||
              (e = cudaMalloc(&d_counts, 2 * sizeof(int))) != cudaSuccess ||
              (e = cudaMemset(s->d_pcell64, 0, pr * sizeof(double))) != cudaSuccess ||
              (e = cudaMemset(s->d_pcell2_64, 0, p2 * sizeof(double))) != cudaSuccess ||
              (e = cudaMemset(s->d_dinit64, 0, di * sizeof(double))) != cudaSuccess ||
              (e = cudaMemset(d_counts, 0, 2 * sizeof(int))) != cudaSuccess))
    rc = cuda_fail(e, "device setup buffers");
  int counts[2] = {0, 0};
  if (!rc && (rc = mbs::setup_cells2(d_slots, s->d_mat, s->d_qslot, d_jit, nx, s->off, ld, dt, s->d_pcell64,
                                     s->d_pcell2_64, s->d_dinit64, d_counts, nullptr)))
    rc = cuda_fail((cudaError_t)rc, "device setup");
  if (!rc && (e = cudaMemcpy(counts, d_counts, sizeof(counts), cudaMemcpyDeviceToHost)) != cudaSuccess)
    rc = cuda_fail(e, "device setup");
  cudaFree(d_slots);
  cudaFree(d_jit);
  cudaFree(d_counts);
  if (rc) return rc;
  if (counts[0]) return fail(MBS_E_NUMERIC, "non-finite per-cell propagator");
  s->has_b2 = counts[1] == 0;
  if (!s->has_b2) {
    cudaFree(s->d_pcell2_64);
    s->d_pcell2_64 = nullptr;
  }
  return 0;
}

int mbs_scenario(mbs_device_t dev, double dt_or_0, double courant, double t_end, long long n_steps,
                 const mbs_source *src, int n_src, const mbs_probe *probes, int n_probes, mbs_scenario_t *out) {
  g_err.clear();
  if (!out) return fail(MBS_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!dev) return fail(MBS_E_INVALID, "device is NULL");
  if (n_src < 0 || n_src > mbs::MAXSRC || (n_src && !src)) return fail(MBS_E_INVALID, "0..%d sources", mbs::MAXSRC);
  if (n_probes < 0 || n_probes > mbs::MAXPROBE || (n_probes && !probes))
    return fail(MBS_E_INVALID, "0..%d probes", mbs::MAXPROBE);
  const int nx = dev->nx;
  const double dz = dev->dz;
  double cmax = 0;   // over the materials that some cell holds
  {
    std::vector<char> used(dev->mats.size(), 0);
    for (int m = 0; m < nx; ++m) used[dev->cell_mat[m]] = 1;
    for (size_t i = 0; i < used.size(); ++i)
      if (used[i]) cmax = std::max(cmax, light_speed(dev->mats[i]));
  }
  double dt;
  if (dt_or_0 > 0) {
    dt = dt_or_0;
    if (dt > dz / cmax * (1 + 1e-12)) return fail(MBS_E_INVALID, "dt exceeds the Courant limit dz / c_max");
  } else {
    if (!(courant > 0 && courant <= 1)) return fail(MBS_E_INVALID, "courant must be in (0, 1]");
    dt = courant * dz / cmax;
  }
  long long nt = n_steps > 0 ? n_steps : (long long)std::ceil(t_end / dt);
  if (nt < 1) return fail(MBS_E_INVALID, "no time steps (t_end <= 0 and n_steps <= 0)");
  if (nt > (1LL << 31)) return fail(MBS_E_INVALID, "too many steps");

  auto s = std::make_unique<mbs_scenario_s>();
  s->dev = dev;
  s->dt = dt;
  s->nt = nt;
  const int N = std::max(dev->N, 2);
  s->N = N;
  s->K = N * N - 1;
  s->P = N * (N - 1) / 2;
  const int K = s->K, P = s->P, N2 = N * N;
  s->ld = ((nx + 2 * mbs::PAD) + 31) / 32 * 32;
  const int n_mat = (int)dev->mats.size();
  const double eta0 = std::sqrt(kMu0 / kEps0);

  // EM coefficients (normalised H^ = eta0 H); the extra last material is the
  // inert pad outside the domain
  s->emc.assign((size_t)(n_mat + 1) * 4, 0.0);
  for (int i = 0; i < n_mat; ++i) {
    const MatDesc &m = dev->mats[i];
    const double eps = kEps0 * m.eps_r, k = dt * m.sigma / (2 * eps);
    s->emc[i * 4 + 0] = (1 - k) / (1 + k) - 1.0;   // a' - 1 (exactly 0 without loss)
    s->emc[i * 4 + 1] = (dt / eps) / (1 + k) / (dz * eta0);
    s->emc[i * 4 + 2] = dt * eta0 / (dz * kMu0 * m.mu_r);
  }
  // slots: one per material with a quantum description
  s->qslot.assign(n_mat + 1, -1);
  std::vector<int> slot_mat;
  for (int i = 0; i < n_mat; ++i)
    if (dev->mats[i].qm >= 0) {
      s->qslot[i] = (int)slot_mat.size();
      slot_mat.push_back(i);
    }
  s->n_slot = (int)slot_mat.size();
  s->qstride = mbs::q_stride(N);
  s->qpar.assign((size_t)std::max(1, s->n_slot) * s->qstride, 0.0);
  s->zref.assign((size_t)std::max(1, s->n_slot) * N2, 0.0);
  std::vector<Step> steps(s->n_slot);
  for (int sl = 0; sl < s->n_slot; ++sl) {
    const MatDesc &m = dev->mats[slot_mat[sl]];
    const QDesc &q = dev->qms[m.qm];
    Step &st = steps[sl];
    build_step(q, 1.0, dt, st);
    const double bp = (dt / (kEps0 * m.eps_r)) / (1 + dt * m.sigma / (2 * kEps0 * m.eps_r));
    const double cpl = bp * m.overlap * q.n3d;
    double *blk = &s->qpar[(size_t)sl * s->qstride];
    for (int i = 0; i < K * K; ++i) blk[i] = st.AKm1[i];
    for (int i = 0; i < K; ++i) {
      blk[K * K + i] = st.c[i];
      blk[K * K + K + i] = cpl * st.g[i];
    }
    blk[K * K + 2 * K] = cpl * st.g0;
    int p = 0;
    for (int j = 0; j < N; ++j)
      for (int k = j + 1; k < N; ++k, ++p) {
        blk[K * K + 2 * K + 1 + p] = (q.lambda[j] - q.lambda[k]) * dt / kHbar;
        blk[K * K + 2 * K + 1 + P + 2 * p] = q.yref[N + 2 * p];
        blk[K * K + 2 * K + 1 + P + 2 * p + 1] = q.yref[N + 2 * p + 1];
      }
    std::copy(q.yref.begin(), q.yref.end(), &s->zref[(size_t)sl * N2]);
  }

  for (double v : s->qpar)
    if (!std::isfinite(v)) return fail(MBS_E_NUMERIC, "non-finite step operator (check H0, mu, rates and dt)");
  if (N >= 4 && s->n_slot == 1) {
    s->tcw.resize(mbs::tc_weight_table(N, s->qpar.data(), nullptr));
    mbs::tc_weight_table(N, s->qpar.data(), s->tcw.data());
  }

  // per-cell state and (jittered media) per-cell step operators; those of
  // jittered two-level media are formed on the device (mbs_setup_dev.cu) at
  // the end, unless MBS_HOST_SETUP is set to a non-empty value other than 0
  const int ld = s->ld, off = s->off;
  s->has_pcell = !dev->jitter.empty() && s->n_slot > 0;
  const char *hs = std::getenv("MBS_HOST_SETUP");
  const bool dev_setup = N == 2 && s->has_pcell && !(hs && hs[0] && std::strcmp(hs, "0") != 0);
  if (!dev_setup) {
    s->Dinit.assign((size_t)K * ld, 0.0);
    if (s->has_pcell) s->pcell.assign((size_t)mbs::pc_rows(N) * ld, 0.0);
  }
  std::vector<double> d0_slot((size_t)std::max(1, s->n_slot) * K, 0.0);
  for (int sl = 0; sl < s->n_slot; ++sl) {
    const QDesc &q = dev->qms[dev->mats[slot_mat[sl]].qm];
    // x^0 - yref = (exp(L0 dt/2) - I) yinit + (yinit - yref)
    std::vector<double> x0(N2, 0.0);
    for (int i = 0; i < N2; ++i)
      for (int j = 0; j < N2; ++j) x0[i] += steps[sl].Ehm1[i * N2 + j] * q.yinit[j];
    for (int i = 0; i < K; ++i) d0_slot[sl * K + i] = x0[full_of(N, i)] + (q.yinit[full_of(N, i)] - q.yref[full_of(N, i)]);
  }
  // structured two-level rows (see bloch2_rows): of jittered media formed in
  // the per-cell loop below, of uniform media from their slots after it
  const bool b2_try = N == 2 && s->n_slot > 0 && !dev_setup;
  if (b2_try) s->pcell2.assign((size_t)7 * ld, 0.0);
  int bad = 0, bad2 = 0;
#pragma omp parallel reduction(+ : bad, bad2) if (!dev_setup)
  if (!dev_setup) {
  Step st;   // one per thread: its vectors keep their capacity from cell to cell
#pragma omp for schedule(dynamic, 256)
  for (int m = 0; m < nx; ++m) {
    const int mt = dev->cell_mat[m];
    const int sl = s->qslot[mt];
    if (sl < 0) continue;
    if (!s->has_pcell) {
      for (int i = 0; i < K; ++i) s->Dinit[(size_t)i * ld + off + m] = d0_slot[sl * K + i];
      continue;
    }
    const MatDesc &mm = dev->mats[mt];
    const QDesc &q = dev->qms[mm.qm];
    const double fd = dev->jitter[2 * m], fh = dev->jitter[2 * m + 1];
    build_step(q, fh, dt, st);
    const double bp = (dt / (kEps0 * mm.eps_r)) / (1 + dt * mm.sigma / (2 * kEps0 * mm.eps_r));
    const double cpl = bp * mm.overlap * q.n3d * fd;
    const size_t col = (size_t)off + m;
    for (int i = 0; i < K * K; ++i) s->pcell[(size_t)i * ld + col] = st.AKm1[i];
    for (int i = 0; i < K; ++i) {
      s->pcell[(size_t)(K * K + i) * ld + col] = st.c[i];
      s->pcell[(size_t)(K * K + K + i) * ld + col] = cpl * st.g[i];
    }
    s->pcell[(size_t)(K * K + 2 * K) * ld + col] = cpl * st.g0;
    if (b2_try) {
      const double w[3] = {cpl * st.g[0], cpl * st.g[1], cpl * st.g[2]};
      double rows[7];
      if (mbs_math::bloch2_rows(st.AKm1.data(), st.c.data(), w, cpl * st.g0, rows))
        for (int r = 0; r < 7; ++r) s->pcell2[(size_t)r * ld + col] = rows[r];
      else
        ++bad2;
    }
    double x0[mbs::NMAX * mbs::NMAX];
    for (int i = 0; i < N2; ++i) {
      x0[i] = 0.0;
      for (int j = 0; j < N2; ++j) x0[i] += st.Ehm1[i * N2 + j] * q.yinit[j];
    }
    for (int i = 0; i < K; ++i)
      s->Dinit[(size_t)i * ld + col] = x0[full_of(N, i)] + (q.yinit[full_of(N, i)] - q.yref[full_of(N, i)]);
    if (!std::isfinite(st.AK[0])) ++bad;
  }
  }
  if (bad) return fail(MBS_E_NUMERIC, "non-finite per-cell propagator");

  if (b2_try && !s->has_pcell) {   // uniform media: one set of rows per slot
    const int stride = s->qstride;
    std::vector<double> srows((size_t)s->n_slot * 7);
    for (int sl = 0; sl < s->n_slot; ++sl) {
      const double *blk = &s->qpar[(size_t)sl * stride];
      if (!mbs_math::bloch2_rows(blk, blk + 9, blk + 12, blk[15], &srows[(size_t)sl * 7])) ++bad2;
    }
    if (bad2 == 0)
#pragma omp parallel for schedule(static)
      for (int m = 0; m < nx; ++m) {
        const int sl = s->qslot[dev->cell_mat[m]];
        if (sl < 0) continue;
        for (int r = 0; r < 7; ++r) s->pcell2[(size_t)r * ld + off + m] = srows[(size_t)sl * 7 + r];
      }
  }
  if (b2_try) {
    s->has_b2 = bad2 == 0;
    if (!s->has_b2) s->pcell2.clear();
  }
  // sources
  for (int k = 0; k < n_src; ++k) {
    const mbs_source &sr = src[k];
    if (sr.kind < 0 || sr.kind > 2) return fail(MBS_E_INVALID, "source %d: bad kind", k);
    if (sr.shape != MBS_SHAPE_SECH && sr.shape != MBS_SHAPE_GAUSS) return fail(MBS_E_INVALID, "source %d: bad shape", k);
    if (sr.cell < 2 || sr.cell > nx - 3) return fail(MBS_E_INVALID, "source %d: cell must be in [2, n_cells-3]", k);
    if (!(sr.tau > 0)) return fail(MBS_E_INVALID, "source %d: tau must be > 0", k);
    if (!std::isfinite(sr.e0) || !std::isfinite(sr.tau) || !std::isfinite(sr.t0) || !std::isfinite(sr.omega) ||
        !std::isfinite(sr.phase))
      return fail(MBS_E_INVALID, "source %d: non-finite parameter", k);
    SrcHost h;
    h.kind = sr.kind;
    h.cell = sr.cell;
    h.face = sr.kind == MBS_SRC_TFSF_RIGHT ? sr.cell : (sr.kind == MBS_SRC_TFSF_LEFT ? sr.cell + 1 : -1);
    h.sH.assign(nt, 0.0);
    h.sE.assign(nt, 0.0);
    const MatDesc &ms = dev->mats[dev->cell_mat[sr.cell]];
    const double cs = light_speed(ms), eta_s = std::sqrt(kMu0 * ms.mu_r / (kEps0 * ms.eps_r));
    const double bh = s->emc[dev->cell_mat[sr.cell] * 4 + 1];
    const double ch = h.face >= 0 ? s->emc[dev->cell_mat[h.face] * 4 + 2] : 0.0;
    auto S = [&](double t) { return sr.e0 * envelope(sr.shape, (t - sr.t0) / sr.tau) * std::sin(sr.omega * t + sr.phase); };
#pragma omp parallel for schedule(static) if (nt > 16384)
    for (long long n = 0; n < nt; ++n) {
      const double tn = n * dt;
      if (sr.kind == MBS_SRC_HARD) {
        h.sE[n] = S(tn + dt);
      } else {
        h.sH[n] = (sr.kind == MBS_SRC_TFSF_RIGHT ? -1.0 : 1.0) * ch * S(tn);
        h.sE[n] = bh * (eta0 / eta_s) * S(tn + 0.5 * dt + 0.5 * dz / cs);
      }
    }
    s->src.push_back(std::move(h));
  }
  // boundaries
  {
    const double cl = light_speed(dev->mats[dev->cell_mat[0]]), cr = light_speed(dev->mats[dev->cell_mat[nx - 1]]);
    s->kmur_l = (cl * dt - dz) / (cl * dt + dz);
    s->kmur_r = (cr * dt - dz) / (cr * dt + dz);
  }
  // probes
  s->pr_coef.assign((size_t)std::max(1, n_probes) * (K + 1), 0.0);
  for (int k = 0; k < n_probes; ++k) {
    const mbs_probe &p = probes[k];
    if (p.cell < 0 || p.cell >= nx) return fail(MBS_E_INVALID, "probe %d: cell out of range", k);
    if (p.quantity < 0 || p.quantity > 3) return fail(MBS_E_INVALID, "probe %d: bad quantity", k);
    s->pr_cell.push_back(p.cell);
    s->pr_q.push_back(p.quantity);
    if (p.quantity >= 2) {
      const int mt = dev->cell_mat[p.cell], sl = s->qslot[mt];
      if (sl < 0) return fail(MBS_E_INVALID, "probe %d: density matrix requested in a cell without medium", k);
      if (p.i < 0 || p.j < 0 || p.i >= N || p.j >= N) return fail(MBS_E_INVALID, "probe %d: level index", k);
      const QDesc &q = dev->qms[dev->mats[mt].qm];
      Step st;
      build_step(q, dev->jitter.empty() ? 1.0 : dev->jitter[2 * p.cell + 1], dt, st);
      const std::vector<double> h = rho_functional(q, p.i, p.j, p.quantity == MBS_Q_RHO_IM);
      std::vector<double> hA(N2, 0.0);   // Ah^T h
      for (int c = 0; c < N2; ++c)
        for (int r = 0; r < N2; ++r) hA[c] += h[r] * st.Ah[r * N2 + c];
      double h0 = 0;
      for (int c = 0; c < N2; ++c) h0 += hA[c] * q.yref[c];
      double *co = &s->pr_coef[(size_t)k * (K + 1)];
      for (int i = 0; i < K; ++i) co[i] = hA[full_of(N, i)] - (i < N - 1 ? hA[N - 1] : 0.0);
      co[K] = h0;
    }
  }
  // cells for the state check: probes plus a strided sample of media
  {
    size_t n_med = 0;
    for (int m = 0; m < nx; ++m) n_med += s->qslot[dev->cell_mat[m]] >= 0;
    const size_t want = 4096;
    const size_t stride = std::max<size_t>(1, n_med / want);
    size_t i = 0;   // index among the medium cells
    for (int m = 0; m < nx; ++m)
      if (s->qslot[dev->cell_mat[m]] >= 0 && i++ % stride == 0) s->chk_cells.push_back(m);
    for (int c : s->pr_cell) s->chk_cells.push_back(c);
  }

  // device-resident tables shared by both precisions
  cudaError_t e = cudaGetDevice(&s->device_id);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  g_h2d = &s->h2d_bytes;
  std::vector<uint8_t> matpad(ld, (uint8_t)n_mat);
  for (int m = 0; m < nx; ++m) matpad[off + m] = dev->cell_mat[m];
  int rc;
  if ((rc = upload_raw(matpad, &s->d_mat)) || (rc = upload_raw(s->qslot, &s->d_qslot)) ||
      (rc = upload_raw(s->pr_cell, &s->d_pr_cell)) || (rc = upload_raw(s->pr_q, &s->d_pr_q)) ||
      (rc = upload_raw(s->chk_cells, &s->d_chk_cells)) || (rc = upload_raw(s->zref, &s->d_zref))) {
    g_h2d = nullptr;
    free_scenario(s.get());
    return rc;
  }
  g_h2d = nullptr;
  if (dev_setup && (rc = setup_on_device(s.get(), slot_mat, dt))) {
    free_scenario(s.get());
    return rc;
  }
  const size_t nchk = std::max<size_t>(1, s->chk_cells.size());
  if ((e = cudaMalloc(&s->d_flags, 4 * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_chk_min, nchk * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&s->d_chk_tr, nchk * sizeof(double))) != cudaSuccess) {
    free_scenario(s.get());
    return cuda_fail(e, "cudaMalloc");
  }
  *out = s.release();
  return MBS_OK;
}

void mbs_scenario_destroy(mbs_scenario_t s) {
  if (!s) return;
  drop_graphs_of(s);
  free_scenario(s);
  delete s;
}

int mbs_scenario_info(mbs_scenario_t s, double *dt, double *dz, long long *n_steps) {
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (dt) *dt = s->dt;
  if (dz) *dz = s->dev->dz;
  if (n_steps) *n_steps = s->nt;
  return MBS_OK;
}

// Upload the precision's tables on first use and reset the state to the
// initial condition (all asynchronous on `st`).

int mbs_fetch_records(mbs_scenario_t s, int probe, double *out, size_t cap, size_t *n_written) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (probe < 0 || probe >= (int)s->pr_cell.size()) return fail(MBS_E_INVALID, "probe index out of range");
  const size_t n = (size_t)s->nt;
  if (n_written) *n_written = n;
  if (!out) return MBS_OK;
  if (cap < n) return fail(MBS_E_INVALID, "capacity %zu < %zu", cap, n);
  if (s->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  const Bundle &b = s->b[s->solved_prec];
  const double scale = s->pr_q[probe] == MBS_Q_H ? 1.0 / std::sqrt(kMu0 / kEps0) : 1.0;
  cudaError_t e;
  if (s->solved_prec == 0) {
    e = cudaMemcpy(out, (const double *)b.rec + (size_t)probe * n, n * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "fetch");
    s->d2h_bytes += (long long)(n * sizeof(double));
    if (scale != 1.0)
      for (size_t i = 0; i < n; ++i) out[i] *= scale;
  } else {
    std::vector<float> f(n);
    e = cudaMemcpy(f.data(), (const float *)b.rec + (size_t)probe * n, n * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "fetch");
    s->d2h_bytes += (long long)(n * sizeof(float));
    // rho probes: the FP32 record is the deviation from the reference value
    const double base = s->pr_q[probe] >= MBS_Q_RHO_RE ? s->pr_coef[(size_t)probe * (s->K + 1) + s->K] : 0.0;
    for (size_t i = 0; i < n; ++i) out[i] = scale * (double)f[i] + base;
  }
  return MBS_OK;
}

int mbs_scenario_set_field(mbs_scenario_t s, const double *e0, size_t n) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (!e0) {
    s->e_init.clear();
    return MBS_OK;
  }
  if (n != (size_t)s->dev->nx) return fail(MBS_E_INVALID, "the initial field needs n_cells = %d values", s->dev->nx);
  for (size_t m = 0; m < n; ++m)
    if (!std::isfinite(e0[m])) return fail(MBS_E_INVALID, "non-finite initial field at cell %zu", m);
  s->e_init.assign(e0, e0 + n);
  return MBS_OK;
}

int mbs_scenario_tile(mbs_scenario_t s, int *tile_steps) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (s->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  if (tile_steps) *tile_steps = s->tile_used;
  return MBS_OK;
}

int mbs_tile_plan(int n_levels, int tile_cells, int nx, int tile_steps, int *n_tiles) {
  g_err.clear();
  const int T = tile_steps;
  if (n_levels < 2 || n_levels > mbs::NMAX) return fail(MBS_E_INVALID, "n_levels %d outside [2, %d]", n_levels, mbs::NMAX);
  if (nx < 8) return fail(MBS_E_INVALID, "nx must be at least 8");
  if (n_levels >= 4) {
    if (!mbs::tiled_tc_geometry_ok(nx, tile_cells, T))
      return fail(MBS_E_INVALID, "tile_steps %d does not fit %d-cell tensor-core tiles on a %d-cell grid", T,
                  tile_cells, nx);
  } else {
    if (tile_cells != 32 * mbs::tile_warps(n_levels) * mbs::tile_lane_cells(n_levels))
      return fail(MBS_E_INVALID, "tiles of N = %d levels hold %d cells", n_levels,
                  32 * mbs::tile_warps(n_levels) * mbs::tile_lane_cells(n_levels));
    if (T % 4 != 0 || T < 4 || T > mbs::tile_max_steps(n_levels))
      return fail(MBS_E_INVALID, "tile_steps must be a multiple of 4 in [4, %d]", mbs::tile_max_steps(n_levels) / 4 * 4);
  }
  const int own = tile_cells - 2 * T;
  if (n_tiles) *n_tiles = (nx + own - 1) / own;
  return MBS_OK;
}

int mbs_scenario_tile_cells(mbs_scenario_t s, int *tile_cells) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (s->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  if (tile_cells)
    *tile_cells = s->tile_used == 0 ? 0 : s->N >= 4 ? s->tc_cells : 32 * mbs::tile_warps(s->N) * mbs::tile_lane_cells(s->N);
  return MBS_OK;
}

int mbs_scenario_counters(mbs_scenario_t s, long long *h2d_bytes, long long *d2h_bytes, long long *kernel_launches) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (h2d_bytes) *h2d_bytes = s->h2d_bytes;
  if (d2h_bytes) *d2h_bytes = s->d2h_bytes;
  if (kernel_launches) *kernel_launches = s->launches;
  return MBS_OK;
}

int mbs_scenario_stats(mbs_scenario_t s, double *max_trace_dev, double *min_eig, long long *n_steps) {
  g_err.clear();
  if (!s) return fail(MBS_E_INVALID, "scenario is NULL");
  if (s->solved_prec < 0) return fail(MBS_E_STATE, "no solve has run");
  if (max_trace_dev) *max_trace_dev = s->st_trace;
  if (min_eig) *min_eig = s->st_min;
  if (n_steps) *n_steps = s->steps_run;
  return MBS_OK;
}
}  // extern "C"
