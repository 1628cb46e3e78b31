// Serving loop (include/hsma.h, hsma_server_*): Monte Carlo chains resident on the device,
// continuous batching of single-charge-move energy changes, overlapped full energies.
//
// * Residency: one batched Engine holds every admitted chain; chains are admitted in index
//   order while the sum of their device footprints fits the budget, and re-admitted from the
//   host copy of their committed state when another chain is closed.
// * Ordering: a chain has at most one request in flight; its released requests wait in a
//   FIFO, so its results follow its own order whatever the mix.
// * Move requests: all ready move requests of idle chains form one batched k_delta launch on
//   a high-priority stream, followed in the same stream by the commit (k_move_surface,
//   k_move_charge) of the accepted ones; one such batch is in flight at a time.
// * Energy requests: each runs on its own low-priority stream slot (pair kernel over that
//   chain's items with a grid capped at a fraction of the GPU, then k_reduce), so move batches
//   keep finding free SMs beside it.
// * Completion is seen with cudaEventQuery; no device-side waits are involved.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "engine.h"

using hsma::DeltaReq;
using hsma::Engine;
using hsma::SysSpec;

namespace {

double now_s()
{
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct EnergySlot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  int4* items_d = nullptr;
  int2* it5_d = nullptr;
  int* sel_d = nullptr;
  int2* selrng_d = nullptr;
  double* epart_d = nullptr;
  unsigned int* ctr_d = nullptr;
  int4* items_h = nullptr;
  int2* it5_h = nullptr;
  int* sel_h = nullptr;
  int2* selrng_h = nullptr;
  double* energy_h = nullptr;
  int req = -1;
  int chain = -1;
};

}  // namespace

struct hsma_server_t {
  Engine* e = nullptr;
  hsma_params prm;
  std::vector<SysSpec> specs;                  // every chain
  std::vector<std::vector<double>> pos, chg;   // committed host state of every chain
  std::vector<int64_t> n;
  std::vector<size_t> footprint;
  std::vector<int> sys_of;                      // chain -> engine system, or -1
  std::vector<int> chain_of;                    // engine system -> chain
  std::vector<char> closed;
  size_t budget = 0;
  int max_batch = 64, energy_slots = 4;
  double sm_frac = 0.75;
  cudaStream_t sA = nullptr;
  cudaEvent_t evA = nullptr;
  std::vector<EnergySlot> slots;
  int items_cap = 0, it5_cap = 0;
  DeltaReq *dreq_h = nullptr, *mreq_h = nullptr, *mreq_d = nullptr;
  int4* ditems_h = nullptr;
  int2 *dranges_h = nullptr, *mitems_h = nullptr, *mitems_d = nullptr;
  double* de_h = nullptr;
  int ditems_cap = 0, mitems_cap = 0;
  std::vector<std::vector<int4>> it4_of;
  std::vector<std::vector<int2>> it5_of;
  std::string err;
  bool loaded = false;
};

static int serr(hsma_server_t* s, int code, const std::string& msg)
{
  if (s) s->err = msg;
  return code;
}

static int scuda(hsma_server_t* s, cudaError_t e, const char* what)
{
  cudaGetLastError();
  return serr(s, HSMA_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SCK(call)                                \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return scuda(s, e_, #call); \
  } while (0)

static void free_buffers(hsma_server_t* s)
{
  for (auto& sl : s->slots) {
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.ev) cudaEventDestroy(sl.ev);
    cudaFree(sl.items_d);
    cudaFree(sl.it5_d);
    cudaFree(sl.sel_d);
    cudaFree(sl.selrng_d);
    cudaFree(sl.epart_d);
    cudaFree(sl.ctr_d);
    cudaFreeHost(sl.items_h);
    cudaFreeHost(sl.it5_h);
    cudaFreeHost(sl.sel_h);
    cudaFreeHost(sl.selrng_h);
    cudaFreeHost(sl.energy_h);
    sl = EnergySlot();
  }
  cudaFreeHost(s->dreq_h);
  cudaFreeHost(s->mreq_h);
  cudaFreeHost(s->ditems_h);
  cudaFreeHost(s->dranges_h);
  cudaFreeHost(s->mitems_h);
  cudaFreeHost(s->de_h);
  cudaFree(s->mreq_d);
  cudaFree(s->mitems_d);
  s->dreq_h = s->mreq_h = s->mreq_d = nullptr;
  s->ditems_h = nullptr;
  s->dranges_h = s->mitems_h = s->mitems_d = nullptr;
  s->de_h = nullptr;
}

// Build the resident set: the engine holds the admitted chains, built from host state.
static int rebuild(hsma_server_t* s)
{
  Engine* e = s->e;
  std::vector<int64_t> ns;
  std::vector<SysSpec> sp;
  std::vector<double> xyz, q;
  s->chain_of.clear();
  for (size_t c = 0; c < s->specs.size(); ++c) {
    if (s->sys_of[c] < 0) continue;
    s->sys_of[c] = (int)s->chain_of.size();
    s->chain_of.push_back((int)c);
    sp.push_back(s->specs[c]);
    ns.push_back(s->n[c]);
    xyz.insert(xyz.end(), s->pos[c].begin(), s->pos[c].end());
    q.insert(q.end(), s->chg[c].begin(), s->chg[c].end());
  }
  if (sp.empty()) return HSMA_OK;
  e->spec = sp;
  e->max_requests = s->max_batch;
  e->layout_uploaded = false;
  e->drop_graphs();
  int rc = e->set_sizes(ns);
  if (rc) return serr(s, rc, e->err);
  rc = e->build(xyz.data(), q.data(), false);
  if (rc) return serr(s, rc, e->err);
  rc = e->ensure_built();
  if (rc) return serr(s, rc, e->err);
  rc = e->ensure_v();
  if (rc) return serr(s, rc, e->err);
  rc = e->check_status();
  if (rc) return serr(s, rc, e->err);
  // per-system work lists of the pair sum and the reduction
  const size_t nsys = sp.size();
  s->it4_of.assign(nsys, {});
  s->it5_of.assign(nsys, {});
  for (const auto& it : e->L.it4) s->it4_of[it.x].push_back(it);
  for (const auto& it : e->L.it5) s->it5_of[it.x].push_back(it);
  int icap = 1, i5cap = 1;
  for (size_t k = 0; k < nsys; ++k) {
    icap = std::max(icap, (int)s->it4_of[k].size());
    i5cap = std::max(i5cap, (int)s->it5_of[k].size());
  }
  // (re)allocate the buffers sized by the resident set
  free_buffers(s);
  s->items_cap = icap;
  s->it5_cap = i5cap;
  int lo = 0, hi = 0;
  SCK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  SCK(cudaStreamCreateWithPriority(&s->sA, cudaStreamNonBlocking, hi));
  s->slots.resize(s->energy_slots);
  for (auto& sl : s->slots) {
    SCK(cudaStreamCreateWithPriority(&sl.st, cudaStreamNonBlocking, lo));
    SCK(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming));
    SCK(cudaMalloc(&sl.items_d, sizeof(int4) * icap));
    SCK(cudaMalloc(&sl.it5_d, sizeof(int2) * i5cap));
    SCK(cudaMalloc(&sl.sel_d, sizeof(int)));
    SCK(cudaMalloc(&sl.selrng_d, sizeof(int2)));
    SCK(cudaMalloc(&sl.epart_d, 16 * (size_t)i5cap));
    SCK(cudaMalloc(&sl.ctr_d, 2 * sizeof(unsigned int)));
    SCK(cudaMemset(sl.ctr_d, 0, 2 * sizeof(unsigned int)));
    SCK(cudaHostAlloc(&sl.items_h, sizeof(int4) * icap, cudaHostAllocDefault));
    SCK(cudaHostAlloc(&sl.it5_h, sizeof(int2) * i5cap, cudaHostAllocDefault));
    SCK(cudaHostAlloc(&sl.sel_h, sizeof(int), cudaHostAllocDefault));
    SCK(cudaHostAlloc(&sl.selrng_h, sizeof(int2), cudaHostAllocDefault));
    SCK(cudaHostAlloc(&sl.energy_h, 16, cudaHostAllocDefault));
  }
  if (!s->evA) SCK(cudaEventCreateWithFlags(&s->evA, cudaEventDisableTiming));
  const int mb = s->max_batch;
  s->ditems_cap = e->L.ditem_cap;
  s->mitems_cap = e->L.mitem_cap;
  SCK(cudaHostAlloc(&s->dreq_h, sizeof(DeltaReq) * mb, cudaHostAllocDefault));
  SCK(cudaHostAlloc(&s->mreq_h, sizeof(DeltaReq) * mb, cudaHostAllocDefault));
  SCK(cudaHostAlloc(&s->ditems_h, sizeof(int4) * s->ditems_cap, cudaHostAllocDefault));
  SCK(cudaHostAlloc(&s->dranges_h, sizeof(int2) * mb, cudaHostAllocDefault));
  SCK(cudaHostAlloc(&s->mitems_h, sizeof(int2) * s->mitems_cap, cudaHostAllocDefault));
  SCK(cudaHostAlloc(&s->de_h, sizeof(double) * mb, cudaHostAllocDefault));
  SCK(cudaMalloc(&s->mreq_d, sizeof(DeltaReq) * mb));
  SCK(cudaMalloc(&s->mitems_d, sizeof(int2) * s->mitems_cap));
  return HSMA_OK;
}

static int admit(hsma_server_t* s, int* admitted)
{
  size_t used = 0;
  int count = 0;
  for (size_t c = 0; c < s->specs.size(); ++c) {
    s->sys_of[c] = -1;
    if (s->closed[c]) continue;
    if (s->budget == 0 || used + s->footprint[c] <= s->budget) {
      used += s->footprint[c];
      s->sys_of[c] = 0;  // marked resident; rebuild assigns the index
      ++count;
    }
  }
  if (admitted) *admitted = count;
  return rebuild(s);
}

// --- batched move requests ----------------------------------------------------------------
static int launch_moves(hsma_server_t* s, const std::vector<int>& ridx, const hsma_request* reqs)
{
  Engine* e = s->e;
  const int nr = (int)ridx.size();
  int ni = 0, nacc = 0, nmi = 0;
  for (int r = 0; r < nr; ++r) {
    const hsma_request& q = reqs[ridx[r]];
    DeltaReq d;
    d.sys = s->sys_of[q.chain];
    d.k = (int)q.k;
    d.x = q.x[0];
    d.y = q.x[1];
    d.z = q.x[2];
    s->dreq_h[r] = d;
    const hsma::SysDev& sd = e->L.sd[d.sys];
    s->dranges_h[r].x = ni;
    for (int b = 0; b < (sd.n + hsma::kDeltaBlock - 1) / hsma::kDeltaBlock; ++b) s->ditems_h[ni++] = make_int4(r, 0, b, 0);
    for (int b = 0; b < (sd.M + hsma::kDeltaBlock - 1) / hsma::kDeltaBlock; ++b) s->ditems_h[ni++] = make_int4(r, 1, b, 0);
    s->dranges_h[r].y = ni - s->dranges_h[r].x;
    if (q.accept) {
      s->mreq_h[nacc] = d;
      for (int b = 0; b < (sd.M + hsma::kDeltaBlock - 1) / hsma::kDeltaBlock; ++b)
        s->mitems_h[nmi++] = make_int2(nacc, b);
      ++nacc;
    }
  }
  SCK(cudaMemcpyAsync(e->dreq_d, s->dreq_h, sizeof(DeltaReq) * nr, cudaMemcpyHostToDevice, s->sA));
  SCK(cudaMemcpyAsync(e->ditems_d, s->ditems_h, sizeof(int4) * ni, cudaMemcpyHostToDevice, s->sA));
  SCK(cudaMemcpyAsync(e->dreqit_d, s->dranges_h, sizeof(int2) * nr, cudaMemcpyHostToDevice, s->sA));
  hsma::launch_delta(e->sys_d, e->ditems_d, ni, e->dreqit_d, e->dreq_d, nr, e->xyz_d, e->q_d, e->perm_d, e->iperm_d,
                     e->srchi_d, e->srclo_d, e->src64_d, e->surfx_d, e->surfqd_d, e->vsurf_d, e->Mn_d, e->tables(),
                     e->dpart_d, e->de_d, e->ctr_delta_d, e->status_d, s->sA);
  SCK(cudaGetLastError());
  SCK(cudaMemcpyAsync(s->de_h, e->de_d, 8 * nr, cudaMemcpyDeviceToHost, s->sA));
  if (nacc > 0) {
    SCK(cudaMemcpyAsync(s->mreq_d, s->mreq_h, sizeof(DeltaReq) * nacc, cudaMemcpyHostToDevice, s->sA));
    SCK(cudaMemcpyAsync(s->mitems_d, s->mitems_h, sizeof(int2) * nmi, cudaMemcpyHostToDevice, s->sA));
    hsma::launch_move(e->sys_d, s->mitems_d, nmi, s->mreq_d, nacc, e->tables(), e->L.maxP, e->xyz_d, e->q_d,
                      e->Mn_d, e->coef_d, e->coef2_d, e->r0_d, e->surfx_d, e->surfqd_d, e->vsurf_d, 1, e->surfa_d,
                      e->surfb_d, e->surf64a_d, e->surf64b_d, e->iperm_d, e->srchi_d, e->srclo_d, e->src64_d,
                      e->boxes_d, s->sA);
    SCK(cudaGetLastError());
    e->launches += nmi > 0 ? 2 : 1;
    // committed state on the host
    for (int r = 0; r < nr; ++r) {
      const hsma_request& q = reqs[ridx[r]];
      if (!q.accept) continue;
      auto& p = s->pos[q.chain];
      p[3 * q.k] = q.x[0];
      p[3 * q.k + 1] = q.x[1];
      p[3 * q.k + 2] = q.x[2];
    }
  }
  e->launches += 1;
  e->pot_ready = false;
  SCK(cudaEventRecord(s->evA, s->sA));
  return HSMA_OK;
}

// --- one full-energy request on a slot ------------------------------------------------------
static int launch_energy(hsma_server_t* s, EnergySlot& sl, int chain)
{
  Engine* e = s->e;
  const int sys = s->sys_of[chain];
  const auto& it4 = s->it4_of[sys];
  const auto& it5 = s->it5_of[sys];
  std::copy(it4.begin(), it4.end(), sl.items_h);
  for (size_t k = 0; k < it5.size(); ++k) sl.it5_h[k] = it5[k];
  sl.sel_h[0] = sys;
  sl.selrng_h[0] = make_int2(0, (int)it5.size());
  SCK(cudaMemcpyAsync(sl.items_d, sl.items_h, sizeof(int4) * it4.size(), cudaMemcpyHostToDevice, sl.st));
  SCK(cudaMemcpyAsync(sl.it5_d, sl.it5_h, sizeof(int2) * it5.size(), cudaMemcpyHostToDevice, sl.st));
  SCK(cudaMemcpyAsync(sl.sel_d, sl.sel_h, sizeof(int), cudaMemcpyHostToDevice, sl.st));
  SCK(cudaMemcpyAsync(sl.selrng_d, sl.selrng_h, sizeof(int2), cudaMemcpyHostToDevice, sl.st));
  SCK(cudaMemsetAsync(sl.ctr_d, 0, sizeof(unsigned int), sl.st));
  if (!it4.empty()) {
    const int occ = e->prec == HSMA_FP64 ? e->occ_f64 : e->occ_f32[e->L.cfg];
    const int cap = std::max(1, (int)std::floor(s->sm_frac * e->num_sms * std::max(occ, 1)));
    const int grid = std::max(1, std::min((int)it4.size(), cap));
    const hsma::PairWork w{sl.items_d, (int)it4.size(), sl.ctr_d, std::min(grid, (int)it4.size())},
        none{nullptr, 0, nullptr, 0};
    if (e->prec == HSMA_FP64)
      hsma::launch_pairs_f64(grid, e->sys_d, w, none, e->src64_d, e->surf64a_d, e->surf64b_d, e->part64_d, sl.st);
    else
      hsma::launch_pairs_f32(e->L.cfg, grid, e->sys_d, w, none, e->srchi_d, e->srclo_d, e->surfa_d, e->surfb_d,
                             e->boxes_d, e->part_d, sl.st);
    e->launches += 1;
  }
  if (!it5.empty()) {
    hsma::launch_reduce(e->sys_d, sl.sel_d, sl.selrng_d, 1, sl.it5_d, (int)it5.size(), e->part_d, e->part64_d, e->prec,
                        e->q_d, e->perm_d, e->r0_d, e->phic_d, e->phir_d, e->phit_d, sl.epart_d, e->energy_d, sl.ctr_d + 1,
                        e->status_d, nullptr, sl.st);
    e->launches += 1;
  }
  SCK(cudaGetLastError());
  SCK(cudaMemcpyAsync(sl.energy_h, e->energy_d + 2 * (size_t)sys, 16, cudaMemcpyDeviceToHost, sl.st));
  SCK(cudaEventRecord(sl.ev, sl.st));
  return HSMA_OK;
}

extern "C" {

int hsma_server_create(int nchains, const double* a, const double* eps1, const double* eps2, const double* kappa,
                       const hsma_params* params, size_t hbm_budget_bytes, int max_batch, int energy_slots,
                       double energy_sm_frac, hsma_server_t** out)
{
  if (!out || nchains <= 0 || !a || !eps1 || !eps2 || !kappa || !params || max_batch < 1 || energy_slots < 1 ||
      !(energy_sm_frac > 0.0) || energy_sm_frac > 1.0)
    return HSMA_E_INVALID_ARG;
  *out = nullptr;
  hsma_server_t* s = new hsma_server_t();
  s->prm = *params;
  s->prm.stream = nullptr;
  for (int c = 0; c < nchains; ++c) {
    SysSpec sp;
    std::string why;
    int rc = hsma::make_spec(a[c], eps1[c], eps2[c], kappa[c], params, &sp, why);
    if (rc) {
      delete s;
      return rc;
    }
    s->specs.push_back(sp);
  }
  s->budget = hbm_budget_bytes;
  s->max_batch = max_batch;
  s->energy_slots = energy_slots;
  s->sm_frac = energy_sm_frac;
  s->e = new Engine();
  s->e->spec = {s->specs[0]};
  int rc = s->e->init(params->device, nullptr, params->precision);
  if (rc) {
    delete s->e;
    delete s;
    return rc;
  }
  *out = s;
  return HSMA_OK;
}

void hsma_server_destroy(hsma_server_t* s)
{
  if (!s) return;
  if (s->e) cudaSetDevice(s->e->device);
  cudaDeviceSynchronize();
  free_buffers(s);
  if (s->sA) cudaStreamDestroy(s->sA);
  if (s->evA) cudaEventDestroy(s->evA);
  delete s->e;
  delete s;
}

const char* hsma_server_last_error(const hsma_server_t* s) { return s ? s->err.c_str() : "NULL server"; }

int hsma_server_load(hsma_server_t* s, const int64_t* n, const double* xyz, const double* q, int* admitted)
{
  if (!s || !n) return HSMA_E_INVALID_ARG;
  const size_t nc = s->specs.size();
  s->n.assign(n, n + nc);
  s->pos.assign(nc, {});
  s->chg.assign(nc, {});
  s->footprint.assign(nc, 0);
  s->sys_of.assign(nc, -1);
  s->closed.assign(nc, 0);
  int64_t off = 0;
  for (size_t c = 0; c < nc; ++c) {
    if (n[c] < 0 || n[c] > (int64_t)INT32_MAX / 4) return serr(s, HSMA_E_INVALID_ARG, "bad sizes");
    if (n[c] > 0 && (!xyz || !q)) return serr(s, HSMA_E_INVALID_ARG, "NULL xyz or q");
    const double a = s->specs[c].a;
    for (int64_t i = off; i < off + n[c]; ++i) {
      const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
      if (!(x * x + y * y + z * z < a * a) || !std::isfinite(q[i]))
        return serr(s, HSMA_E_OUTSIDE, "a charge lies outside its cavity");
    }
    s->pos[c].assign(xyz + 3 * off, xyz + 3 * (off + n[c]));
    s->chg[c].assign(q + off, q + off + n[c]);
    // device footprint of the chain on its own
    Engine& e = *s->e;
    e.spec = {s->specs[c]};
    s->footprint[c] = e.make_layout({n[c]}, e.prec == HSMA_FP64 ? 0 : e.choose_config({n[c]})).bytes;
    off += n[c];
  }
  int rc = admit(s, admitted);
  if (rc) return rc;
  s->loaded = true;
  return HSMA_OK;
}

int hsma_server_close_chain(hsma_server_t* s, int c, int* admitted)
{
  if (!s || !s->loaded || c < 0 || c >= (int)s->specs.size()) return serr(s, HSMA_E_INVALID_ARG, "bad chain");
  cudaDeviceSynchronize();
  s->closed[c] = 1;
  return admit(s, admitted);
}

int hsma_server_positions(hsma_server_t* s, int c, double* xyz_out, int64_t n)
{
  if (!s || !s->loaded || c < 0 || c >= (int)s->specs.size() || !xyz_out || n != s->n[c])
    return serr(s, HSMA_E_INVALID_ARG, "bad arguments");
  std::copy(s->pos[c].begin(), s->pos[c].end(), xyz_out);
  return HSMA_OK;
}

int hsma_server_run(hsma_server_t* s, int nreq, const hsma_request* reqs, hsma_result* results)
{
  if (!s || nreq < 0 || (nreq > 0 && (!reqs || !results))) return serr(s, HSMA_E_INVALID_ARG, "bad arguments");
  if (!s->loaded) return serr(s, HSMA_E_STATE, "no chains loaded");
  Engine* e = s->e;
  SCK(cudaSetDevice(e->device));
  SCK(cudaDeviceSynchronize());
  const int nc = (int)s->specs.size();
  std::vector<int> order(nreq);
  for (int r = 0; r < nreq; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return reqs[x].t_arrival < reqs[y].t_arrival; });
  std::vector<std::deque<int>> fifo(nc);
  std::vector<char> busy(nc, 0);
  for (int r = 0; r < nreq; ++r) {
    results[r].id = reqs[r].id;
    results[r].status = HSMA_E_STATE;
    results[r].value = 0.0;
    results[r].t_arrival = reqs[r].t_arrival;
    results[r].t_done = -1.0;
  }
  int next = 0, done = 0;
  std::vector<int> batch;  // request indices in the move batch in flight
  bool batch_live = false;
  const double t0 = now_s();
  while (done < nreq) {
    const double t = now_s() - t0;
    // release arrived requests
    while (next < nreq && reqs[order[next]].t_arrival <= t) {
      const int r = order[next++];
      const hsma_request& q = reqs[r];
      int st = HSMA_OK;
      if (q.chain < 0 || q.chain >= nc)
        st = HSMA_E_INVALID_ARG;
      else if (s->sys_of[q.chain] < 0)
        st = HSMA_E_BUSY;
      else if (q.kind == HSMA_REQ_DELTA) {
        const double a = s->specs[q.chain].a;
        const double r2 = q.x[0] * q.x[0] + q.x[1] * q.x[1] + q.x[2] * q.x[2];
        if (q.k < 0 || q.k >= s->n[q.chain]) st = HSMA_E_INVALID_ARG;
        else if (!(r2 < a * a) || !std::isfinite(r2)) st = HSMA_E_OUTSIDE;
      } else if (q.kind != HSMA_REQ_ENERGY) {
        st = HSMA_E_INVALID_ARG;
      }
      if (st != HSMA_OK) {
        results[r].status = st;
        results[r].t_done = now_s() - t0;
        ++done;
        continue;
      }
      fifo[q.chain].push_back(r);
    }
    bool progress = false;
    // completions
    if (batch_live) {
      const cudaError_t qe = cudaEventQuery(s->evA);
      if (qe == cudaSuccess) {
        const double td = now_s() - t0;
        for (size_t i = 0; i < batch.size(); ++i) {
          const int r = batch[i];
          results[r].status = HSMA_OK;
          results[r].value = s->de_h[i];
          results[r].t_done = td;
          busy[reqs[r].chain] = 0;
          ++done;
        }
        batch.clear();
        batch_live = false;
        progress = true;
      } else if (qe != cudaErrorNotReady) {
        return scuda(s, qe, "move batch");
      }
    }
    for (auto& sl : s->slots) {
      if (sl.req < 0) continue;
      const cudaError_t qe = cudaEventQuery(sl.ev);
      if (qe == cudaSuccess) {
        results[sl.req].status = HSMA_OK;
        results[sl.req].value = sl.energy_h[0];
        results[sl.req].t_done = now_s() - t0;
        busy[sl.chain] = 0;
        ++done;
        sl.req = -1;
        sl.chain = -1;
        progress = true;
      } else if (qe != cudaErrorNotReady) {
        return scuda(s, qe, "energy request");
      }
    }
    // issue: one move batch of every idle chain whose next request is a move
    if (!batch_live) {
      for (int c = 0; c < nc && (int)batch.size() < s->max_batch; ++c) {
        if (busy[c] || fifo[c].empty()) continue;
        const int r = fifo[c].front();
        if (reqs[r].kind != HSMA_REQ_DELTA) continue;
        fifo[c].pop_front();
        busy[c] = 1;
        batch.push_back(r);
      }
      if (!batch.empty()) {
        int rc = launch_moves(s, batch, reqs);
        if (rc) return rc;
        batch_live = true;
        progress = true;
      }
    }
    // issue: full energies into free slots (oldest first)
    for (auto& sl : s->slots) {
      if (sl.req >= 0) continue;
      int best = -1, bc = -1;
      for (int c = 0; c < nc; ++c) {
        if (busy[c] || fifo[c].empty()) continue;
        const int r = fifo[c].front();
        if (reqs[r].kind != HSMA_REQ_ENERGY) continue;
        if (best < 0 || reqs[r].t_arrival < reqs[best].t_arrival) {
          best = r;
          bc = c;
        }
      }
      if (best < 0) break;
      fifo[bc].pop_front();
      busy[bc] = 1;
      sl.req = best;
      sl.chain = bc;
      int rc = launch_energy(s, sl, bc);
      if (rc) return rc;
      progress = true;
    }
    (void)progress;
  }
  SCK(cudaDeviceSynchronize());
  int st = 0;
  SCK(cudaMemcpy(&st, e->status_d, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    cudaMemset(e->status_d, 0, sizeof(int));
    return serr(s, (st & hsma::kStNonFinite) ? HSMA_E_NONFINITE : HSMA_E_OUTSIDE, "device status flagged");
  }
  return HSMA_OK;
}

}  // extern "C"
