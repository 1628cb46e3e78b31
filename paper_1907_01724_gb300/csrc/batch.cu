// C ABI of the batched engine (include/hsma.h, hsma_batch_*) and the pair-tile autotuner.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"

using hsma::DeltaReq;
using hsma::Engine;

struct hsma_batch_t {
  Engine* e = nullptr;
  std::vector<int64_t> n;
  std::string err;
};

namespace hsma {

// Time every pair configuration on the current inputs and keep the fastest for this size class:
// with overlap on, the overlapped build + potential step that a build followed by an evaluation
// runs (the configuration sets the pair items that overlap the coefficient chain); with overlap
// off, the potential pass alone (pair sum plus the reduction of its partials).  The inputs (xyz,
// q) sit before every configuration-dependent buffer of the workspace, so each configuration
// rebuilds its sources from them in place.  A sweep takes the median of reps steps per
// configuration; the kTuneFinal fastest are then timed again in interleaved rounds (one step of
// each per round, 2 reps rounds), so that a drift of the clocks over the sweep does not decide
// between configurations a few percent apart.  With overlap on, the winner is then timed with
// both schedules of the real/Kelvin pair items (beside the moment chain or after it, see
// issue_fused) in interleaved rounds, and the faster schedule is kept with it.
constexpr int kTuneFinal = 3;

int Engine::tune_time_config(int c, int side_mode, int steps, std::vector<float>& t)
{
  forced_cfg = c;
  forced_side = side_mode;
  layout_uploaded = false;
  const std::vector<int64_t> ns = cur_ns;
  int rc = set_sizes(ns);
  if (rc) return rc;
  rc = prepare_inputs();
  if (rc) return rc;
  rc = run_graph(&g_build, &Engine::issue_build);
  if (rc) return rc;
  sources_ready = true;
  build_pending = false;
  for (int r = 0; r < steps + 1; ++r) {
    pot_ready = false;
    float ms = 0.f;
    if (overlap) {
      build_pending = true;
      cudaError_t e = cudaEventRecord(ev_tune0, stream);
      if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord (autotune)");
      rc = potentials();
      if (rc) return rc;
      e = cudaEventRecord(ev_tune1, stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev_tune1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev_tune0, ev_tune1);
      if (e != cudaSuccess) return cuda_fail(e, "timing (autotune)");
    } else {
      rc = potentials();
      if (rc) return rc;
      rc = last_pot_time(&ms);
      if (rc) return rc;
    }
    if (r > 0) t.push_back(ms);  // the first step after a rebuild is a warm-up
  }
  return HSMA_OK;
}

int Engine::autotune(int reps, int* best_out, float* best_ms_out)
{
  if (prec == HSMA_FP64) return fail(HSMA_E_INVALID_ARG, "autotuning applies to the FP32 pair sum");
  if (!sources_ready) return fail(HSMA_E_STATE, "sources have not been built");
  reps = std::max(1, reps);
  const std::vector<int64_t> ns = cur_ns;
  size_t need = 0;
  for (int c = 0; c < pair_config_count(); ++c) need = std::max(need, make_layout(ns, c).bytes);
  if (need > ws_cap && ws_user) return fail(HSMA_E_OOM, "attached workspace too small to autotune");
  if (need > ws_cap) {
    // grow, keeping the inputs (at the same offsets in every layout)
    char* nw = nullptr;
    cudaError_t e = cudaMalloc((void**)&nw, need);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (autotune)");
    e = cudaMemcpyAsync(nw + L.o_xyz, xyz_d, 24 * L.totN, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nw + L.o_q, q_d, 8 * L.totN, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "copy inputs (autotune)");
    if (ws_owned && ws) cudaFree(ws);
    ws = nw;
    ws_cap = need;
    ws_owned = true;
  }
  const int saved_forced = forced_cfg, saved_side = forced_side;
  const int side0 = choose_side(ns);  // the schedule of the sweep (forced, tuned or default)
  auto median = [](std::vector<float>& t) {
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
  };
  std::vector<std::pair<float, int>> sweep;
  for (int c = 0; c < pair_config_count(); ++c) {
    std::vector<float> t;
    int rc = tune_time_config(c, side0, reps, t);
    if (rc) return rc;
    sweep.emplace_back(median(t), c);
  }
  std::sort(sweep.begin(), sweep.end());
  const int nfin = std::min<int>(kTuneFinal, (int)sweep.size());
  std::vector<std::vector<float>> tf(nfin);
  for (int round = 0; round < 2 * reps && nfin > 1; ++round)
    for (int k = 0; k < nfin; ++k) {
      int rc = tune_time_config(sweep[k].second, side0, 1, tf[k]);
      if (rc) return rc;
    }
  int best = sweep[0].second;
  float best_ms = sweep[0].first;
  if (nfin > 1) {
    best_ms = -1.f;
    for (int k = 0; k < nfin; ++k) {
      const float med = median(tf[k]);
      if (best_ms < 0.f || med < best_ms) {
        best = sweep[k].second;
        best_ms = med;
      }
    }
  }
  // the schedule of the real/Kelvin items for the winner (only a forced schedule is kept as is)
  int best_side = side0;
  if (overlap && saved_side < 0) {
    constexpr int kSchedules = 3;
    std::vector<float> ts[kSchedules];
    for (int round = 0; round < 2 * reps; ++round)
      for (int sd = 0; sd < kSchedules; ++sd) {
        int rc = tune_time_config(best, sd, 1, ts[sd]);
        if (rc) return rc;
      }
    best_side = 1;
    best_ms = median(ts[1]);
    for (int sd : {2, 0}) {
      const float m = median(ts[sd]);
      if (m < best_ms) {
        best_ms = m;
        best_side = sd;
      }
    }
  }
  forced_cfg = saved_forced;
  forced_side = saved_side;
  const int bucket = tune_bucket([&] {
    int64_t s = 0;
    for (auto v : ns) s += v;
    return s;
  }(), (int)ns.size());
  bool found = false;
  for (auto& e : tuned)
    if (e.bucket == bucket) {
      e.cfg = best;
      e.side = best_side;
      found = true;
    }
  if (!found) tuned.push_back(Tuned{bucket, best, best_side});
  layout_uploaded = false;
  int rc = set_sizes(ns);
  if (rc) return rc;
  rc = prepare_inputs();
  if (rc) return rc;
  rc = run_graph(&g_build, &Engine::issue_build);
  if (rc) return rc;
  sources_ready = true;
  build_pending = false;
  pot_ready = false;
  v_ready = false;
  if (best_out) *best_out = best;
  if (best_ms_out) *best_ms_out = best_ms;
  return HSMA_OK;
}

}  // namespace hsma

static int berr(hsma_batch_t* b, int code, const char* msg)
{
  if (b) b->err = msg;
  return code;
}

static int bfrom(hsma_batch_t* b, int rc)
{
  if (rc != HSMA_OK) b->err = b->e->err;
  return rc;
}

static bool sizes_ok(const hsma_batch_t* b, const int64_t* n, int64_t* total)
{
  int64_t t = 0;
  for (size_t s = 0; s < b->e->spec.size(); ++s) {
    if (n[s] < 0 || n[s] > (int64_t)INT32_MAX / 4) return false;
    t += n[s];
  }
  if (t > (int64_t)INT32_MAX / 4) return false;
  *total = t;
  return true;
}

extern "C" {

int hsma_batch_create(int nsys, const double* a, const double* eps1, const double* eps2, const double* kappa,
                      const hsma_params* params, hsma_batch_t** out)
{
  if (!out || nsys <= 0 || !a || !eps1 || !eps2 || !kappa || !params) return HSMA_E_INVALID_ARG;
  *out = nullptr;
  std::vector<hsma::SysSpec> specs(nsys);
  for (int s = 0; s < nsys; ++s) {
    std::string why;
    int rc = hsma::make_spec(a[s], eps1[s], eps2[s], kappa[s], params, &specs[s], why);
    if (rc) return rc;
  }
  hsma_batch_t* b = new hsma_batch_t();
  b->e = new Engine();
  b->e->spec = specs;
  int rc = b->e->init(params->device, params->stream, params->precision);
  if (rc) {
    delete b->e;
    delete b;
    return rc;
  }
  *out = b;
  return HSMA_OK;
}

void hsma_batch_destroy(hsma_batch_t* b)
{
  if (!b) return;
  delete b->e;
  delete b;
}

const char* hsma_batch_last_error(const hsma_batch_t* b) { return b ? b->err.c_str() : "NULL handle"; }

int hsma_batch_workspace_size(hsma_batch_t* b, const int64_t* n, size_t* bytes)
{
  if (!b || !n || !bytes) return HSMA_E_INVALID_ARG;
  int64_t tot;
  if (!sizes_ok(b, n, &tot)) return berr(b, HSMA_E_INVALID_ARG, "bad sizes");
  std::vector<int64_t> ns(n, n + b->e->spec.size());
  // the largest layout over all tile configurations, so that a workspace of this size also
  // serves the autotuner
  size_t mx = 0;
  const int ncfg = b->e->prec == HSMA_FP64 ? 1 : hsma::pair_config_count();
  for (int c = 0; c < ncfg; ++c) mx = std::max(mx, b->e->make_layout(ns, c).bytes);
  *bytes = mx;
  return HSMA_OK;
}

int hsma_batch_attach_workspace(hsma_batch_t* b, void* device_ptr, size_t bytes)
{
  if (!b) return HSMA_E_INVALID_ARG;
  b->n.clear();
  return bfrom(b, b->e->attach(device_ptr, bytes));
}

int hsma_batch_set_max_requests(hsma_batch_t* b, int max_requests)
{
  if (!b || max_requests < 1 || max_requests > (1 << 20)) return berr(b, HSMA_E_INVALID_ARG, "bad max_requests");
  b->e->max_requests = max_requests;
  b->e->layout_uploaded = false;
  b->e->sources_ready = false;
  b->e->build_pending = false;
  b->n.clear();
  return HSMA_OK;
}

static int batch_build(hsma_batch_t* b, const int64_t* n, const double* xyz, const double* q, bool dev)
{
  if (!b || !n) return HSMA_E_INVALID_ARG;
  int64_t tot;
  if (!sizes_ok(b, n, &tot)) return berr(b, HSMA_E_INVALID_ARG, "bad sizes");
  if (tot > 0 && (!xyz || !q)) return berr(b, HSMA_E_INVALID_ARG, "NULL xyz or q");
  std::vector<int64_t> ns(n, n + b->e->spec.size());
  // (every charge is checked by the pass's first kernel, k_order_keys, for host and device
  // inputs alike: the evaluation that runs the pass returns HSMA_E_OUTSIDE)
  int rc = b->e->set_sizes(ns);
  if (rc) return bfrom(b, rc);
  b->n = ns;
  return bfrom(b, b->e->build(xyz, q, dev));
}

int hsma_batch_build_sources(hsma_batch_t* b, const int64_t* n, const double* xyz, const double* q)
{
  return batch_build(b, n, xyz, q, false);
}

int hsma_batch_build_sources_device(hsma_batch_t* b, const int64_t* n, const double* xyz_dev, const double* q_dev)
{
  return batch_build(b, n, xyz_dev, q_dev, true);
}

static const double* bpick(Engine* e, int what)
{
  if (what == HSMA_TOTAL) return e->phit_d;
  if (what == HSMA_REACTION) return e->phir_d;
  if (what == HSMA_COULOMB) return e->phic_d;
  return nullptr;
}

static int batch_pot(hsma_batch_t* b, double* phi, int what, bool dev)
{
  if (!b) return HSMA_E_INVALID_ARG;
  if (b->n.empty()) return berr(b, HSMA_E_STATE, "sources have not been built");
  const double* src = bpick(b->e, what);
  if (!src) return berr(b, HSMA_E_INVALID_ARG, "bad 'what'");
  int64_t tot = 0;
  for (auto v : b->n) tot += v;
  if (tot > 0 && !phi) return berr(b, HSMA_E_INVALID_ARG, "NULL phi");
  // a pass run by this call writes the result straight to the caller's device array, or (host
  // output) to pinned staging together with the energy terms (hsma_batch_energy then reads them
  // without a second round trip); a pass already run: copies
  hsma::OutDesc od{dev && tot > 0 ? phi : nullptr, nullptr, nullptr, Engine::out_lane(what), 0};
  double* phi_dev = nullptr;  // a page-locked host output: written by the device itself
  if (!dev) {
    const int rs = b->e->ensure_host_stage(tot);
    if (rs) return bfrom(b, rs);
    phi_dev = static_cast<double*>(const_cast<void*>(hsma::pinned_device_address(phi)));
    od = b->e->host_outputs(tot, what, phi_dev);
  }
  bool wrote = false;
  int rc = b->e->potentials(od, &wrote);
  if (rc) return bfrom(b, rc);
  if (dev) {
    if (tot > 0 && !wrote) {
      cudaError_t e = cudaMemcpyAsync(phi, src, 8 * tot, cudaMemcpyDeviceToDevice, b->e->stream);
      if (e != cudaSuccess) return bfrom(b, b->e->cuda_fail(e, "copy phi"));
    }
    return HSMA_OK;
  }
  return bfrom(b, b->e->copy_to_host(src, tot, phi, wrote, phi_dev != nullptr));
}

static int batch_field(hsma_batch_t* b, double* E, int what, bool dev)
{
  if (!b) return HSMA_E_INVALID_ARG;
  if (b->n.empty()) return berr(b, HSMA_E_STATE, "sources have not been built");
  if (what != HSMA_TOTAL && what != HSMA_REACTION && what != HSMA_COULOMB) return berr(b, HSMA_E_INVALID_ARG, "bad 'what'");
  int64_t tot = 0;
  for (auto v : b->n) tot += v;
  if (tot > 0 && !E) return berr(b, HSMA_E_INVALID_ARG, "NULL E");
  // host output through the pinned staging (with the energies and the status, one round trip)
  int rc = dev ? HSMA_OK : b->e->ensure_host_stage(3 * tot);
  if (rc) return bfrom(b, rc);
  rc = b->e->field();
  if (rc) return bfrom(b, rc);
  const double* src = what == HSMA_TOTAL ? b->e->Et_d : (what == HSMA_REACTION ? b->e->Er_d : b->e->Ec_d);
  if (!dev) return bfrom(b, b->e->copy_to_host(src, 3 * tot, E));
  if (tot > 0) {
    cudaError_t e = cudaMemcpyAsync(E, src, 24 * tot, cudaMemcpyDeviceToDevice, b->e->stream);
    if (e != cudaSuccess) return bfrom(b, b->e->cuda_fail(e, "copy E"));
  }
  return HSMA_OK;
}

int hsma_batch_set_overlap(hsma_batch_t* b, int on)
{
  if (!b) return HSMA_E_INVALID_ARG;
  b->e->overlap = on != 0;
  return HSMA_OK;
}

int hsma_batch_set_pair_schedule(hsma_batch_t* b, int mode)
{
  if (!b || mode < -1 || mode > 2) return berr(b, HSMA_E_INVALID_ARG, "bad schedule");
  if (b->e->forced_side != mode) {
    b->e->forced_side = mode;
    b->e->layout_uploaded = false;  // the next call rebuilds the layout and its graphs
    b->e->sources_ready = false;
    b->e->build_pending = false;
    b->n.clear();
  }
  return HSMA_OK;
}

int hsma_batch_pair_schedule(const hsma_batch_t* b, int* mode)
{
  if (!b || !mode) return HSMA_E_INVALID_ARG;
  *mode = b->e->have_layout ? b->e->rk_side : b->e->choose_side(b->e->cur_ns);
  return HSMA_OK;
}

int hsma_batch_field(hsma_batch_t* b, double* E, int what) { return batch_field(b, E, what, false); }
int hsma_batch_field_device(hsma_batch_t* b, double* E_dev, int what) { return batch_field(b, E_dev, what, true); }

int hsma_batch_potential(hsma_batch_t* b, double* phi, int what) { return batch_pot(b, phi, what, false); }
int hsma_batch_potential_device(hsma_batch_t* b, double* phi_dev, int what)
{
  return batch_pot(b, phi_dev, what, true);
}

int hsma_batch_energy(hsma_batch_t* b, double* e_total, double* e_reaction)
{
  if (!b) return HSMA_E_INVALID_ARG;
  if (b->n.empty()) return berr(b, HSMA_E_STATE, "sources have not been built");
  int rc = b->e->potentials();
  if (rc) return bfrom(b, rc);
  const size_t ns = b->e->spec.size();
  std::vector<double> en(2 * ns);
  // from the pinned mirror when a host-output call of this pass staged it (status checked)
  rc = b->e->read_energies(en.data());
  if (rc) return bfrom(b, rc);
  for (size_t s = 0; s < ns; ++s) {
    if (e_total) e_total[s] = en[2 * s];
    if (e_reaction) e_reaction[s] = en[2 * s + 1];
  }
  return HSMA_OK;
}

static int make_reqs(hsma_batch_t* b, int nreq, const int* sys, const int64_t* k, const double* x,
                     std::vector<DeltaReq>& out)
{
  if (nreq < 0 || (nreq > 0 && (!sys || !k || !x))) return berr(b, HSMA_E_INVALID_ARG, "bad request arrays");
  out.resize(nreq);
  for (int r = 0; r < nreq; ++r) {
    if (k[r] < 0 || k[r] > INT32_MAX) return berr(b, HSMA_E_INVALID_ARG, "charge index out of range");
    out[r].sys = sys[r];
    out[r].k = (int)k[r];
    out[r].x = x[3 * r];
    out[r].y = x[3 * r + 1];
    out[r].z = x[3 * r + 2];
  }
  return HSMA_OK;
}

int hsma_batch_delta_energy(hsma_batch_t* b, int nreq, const int* sys, const int64_t* k, const double* x_new,
                            double* de)
{
  if (!b) return HSMA_E_INVALID_ARG;
  if (nreq > 0 && !de) return berr(b, HSMA_E_INVALID_ARG, "NULL de");
  std::vector<DeltaReq> reqs;
  int rc = make_reqs(b, nreq, sys, k, x_new, reqs);
  if (rc) return rc;
  return bfrom(b, b->e->delta_batch(reqs, de));
}

int hsma_batch_apply_moves(hsma_batch_t* b, int nreq, const int* sys, const int64_t* k, const double* x_new)
{
  if (!b) return HSMA_E_INVALID_ARG;
  std::vector<DeltaReq> reqs;
  int rc = make_reqs(b, nreq, sys, k, x_new, reqs);
  if (rc) return rc;
  return bfrom(b, b->e->move_batch(reqs));
}

int64_t hsma_batch_kernel_launches(const hsma_batch_t* b) { return b ? b->e->launches : 0; }

int hsma_batch_last_pair_time(hsma_batch_t* b, float* ms)
{
  if (!b || !ms) return HSMA_E_INVALID_ARG;
  return bfrom(b, b->e->last_pair_time(ms));
}

int hsma_pair_config_count(void) { return hsma::pair_config_count(); }

int hsma_pair_config_info(int idx, int* threads, int* targets_per_thread, int* items_per_slot)
{
  if (idx < 0 || idx >= hsma::pair_config_count()) return HSMA_E_INVALID_ARG;
  const hsma::PairConfig c = hsma::pair_config(idx);
  if (threads) *threads = c.threads;
  if (targets_per_thread) *targets_per_thread = c.k;
  if (items_per_slot) *items_per_slot = c.items_per_slot;
  return HSMA_OK;
}

int hsma_batch_set_pair_config(hsma_batch_t* b, int cfg)
{
  if (!b || cfg < -1 || cfg >= hsma::pair_config_count()) return berr(b, HSMA_E_INVALID_ARG, "bad configuration");
  b->e->forced_cfg = cfg;
  b->e->layout_uploaded = false;
  b->e->sources_ready = false;
  b->e->build_pending = false;
  b->n.clear();
  return HSMA_OK;
}

int hsma_batch_autotune(hsma_batch_t* b, int reps, int* best, float* best_ms)
{
  if (!b) return HSMA_E_INVALID_ARG;
  return bfrom(b, b->e->autotune(reps, best, best_ms));
}

}  // extern "C"
