// Engine: device state, layout and launch sequencing for one or more HSMA cavity systems.
#pragma once

#include <string>
#include <utility>
#include <vector>

#include <cmath>

#include "hsma_internal.cuh"
#include "tree.h"

namespace hsma {

// Host description of one system (Sec. 2.1 inputs plus the numerical parameters).
struct SysSpec {
  double a, eps1, eps2, kappa, tau, dy_rel, coulk;
  int p, M, F1, F2;
};

int make_spec(double a, double eps1, double eps2, double kappa, const hsma_params* prm, SysSpec* out,
              std::string& why);
int tune_bucket(int64_t total_n, int nsys);
const void* pinned_device_address(const void* p);  // page-locked host memory: its device address

// Sizes, offsets into the workspace, and work lists for a set of systems.
struct Layout {
  std::vector<SysDev> sd;
  std::vector<int2> it12, it2r, it3, it5;
  std::vector<int2> it3m;     // (system, block of kSurfMatWarps surf_pw points) of k_surface_mat
  int surf_pw = 1;            // surface points per warp of k_surface_mat (with the basis)
  std::vector<int2> itsb;     // (representative system, point block) of every surface-basis table
  std::vector<int2> itord;    // (system, block of kOrderBlock charges): spatial order and records
  std::vector<int2> itsort;   // (system, part): the blocks of k_order_sort
  int64_t totBoxes = 0;       // 32-record boxes (real + Kelvin) of all systems
  int momG = 1;               // charges per moment group (k_moments, FP64 path)
  std::vector<int2> itmu;     // FP32 path: moment units (system, tile << 7 | column pair); it12
                              // then holds the prep items (system, block of kMomPrepCharges)
  int64_t totZ = 0;           // FP32 path: slots of the (p+1) x n moment tables of all systems
  bool use_sb = false;        // surface synthesis through the basis tables
  int64_t totSB = 0;          // 8-byte slots of all basis tables
  std::vector<int4> it4;
  std::vector<int4> it4x;     // it4 split: real and Kelvin items first (nRK), then surface items
  int nRK = 0;
  std::vector<int4> it4f;     // items of the field pass (FP32: every (target block, chunk) one way)
  std::vector<int4> it4fx;    // it4f split as it4x
  int nRKf = 0;
  int nw = 1;                 // pair-kernel workers per CTA (FP32: warps)
  int order_smem_n = 4096;    // charges k_order_sort keeps in shared memory (order_smem_charges)
  std::vector<int> sel;       // all systems, in order (energy pass of a full launch)
  std::vector<int2> selrng;   // their reduce-item ranges
  size_t o_sel = 0, o_selrng = 0;
  int cfg = 0, maxP = 1, pmax = 0, mom_stride = 3, pair_grid = 1;
  int64_t totN = 0, totM = 0, totP = 0, totMn = 0, totMom = 0, totPart = 0;
  size_t o_sys = 0, o_Mn = 0, o_rec_a = 0, o_rec_b = 0, o_sect = 0, o_inv_np1 = 0, o_xyz = 0, o_q = 0;
  size_t o_rec_a2 = 0, o_rec_b2 = 0, o_sect2 = 0, o_mtab = 0;
  size_t o_mgeo = 0, o_mz = 0, o_mwq = 0, o_mcen = 0, o_itmu = 0;
  size_t o_src64 = 0, o_surf64a = 0, o_surf64b = 0, o_part64 = 0;
  size_t o_srchi = 0, o_srclo = 0, o_surfa = 0, o_surfb = 0, o_part = 0;
  size_t o_surfx = 0, o_surfqd = 0, o_vsurf = 0;
  int max_req = 1, ditem_cap = 1, mitem_cap = 1;
  size_t o_dreq = 0, o_ditems = 0, o_dreqit = 0, o_mitems = 0, o_dpart = 0, o_de = 0;
  size_t o_sb = 0, o_coef2 = 0, o_itsb = 0;
  size_t o_perm = 0, o_iperm = 0, o_key = 0, o_hist = 0, o_sortscr = 0, o_xs = 0, o_boxes = 0, o_itord = 0, o_itsort = 0;
  size_t o_redctr = 0;
  size_t o_mom = 0, o_coef = 0, o_r0 = 0, o_phic = 0, o_phir = 0, o_phit = 0, o_epart = 0, o_energy = 0, o_ctr = 0, o_outdesc = 0, o_indesc = 0;
  size_t o_it3m = 0;
  size_t o_it12 = 0, o_it2r = 0, o_it3 = 0, o_it5 = 0, o_it4 = 0, o_it4x = 0, o_it4f = 0, o_it4fx = 0;
  // far-field tree (one FP32 system, Engine::far_theta > 0): node levels, order, and its arrays;
  // the pair kernel then takes only the surface items and chunks 0 / 1 are the tree's sums
  bool tree = false;
  int tL = 0, tP = 0;
  size_t o_tnode = 0, o_tgeo = 0, o_tbox = 0, o_tmom = 0, o_tfarp = 0, o_tfarL = 0, o_tctr = 0;
  size_t bytes = 0;
};

class Engine {
 public:
  ~Engine();
  int init(int dev, void* user_stream, int precision);
  Layout make_layout(const std::vector<int64_t>& ns, int cfg) const;
  int set_sizes(const std::vector<int64_t>& ns);
  int attach(void* ptr, size_t bytes);
  int build(const double* xyz, const double* q, bool device_inputs);
  // a potential pass if the potentials are not current; od: where it also writes its results
  // (OutDesc), *wrote: whether a pass ran (and so wrote them)
  int potentials(const OutDesc& od = OutDesc{nullptr, nullptr, nullptr, 0, 0}, bool* wrote = nullptr);
  int set_outputs(const OutDesc& od);
  OutDesc* outdesc_d = nullptr;
  // Inputs of the next build pass (InDesc in the workspace): the caller's device arrays while a
  // build from them is pending (the pass reads them in place and copies them to xyz_d, q_d),
  // else xyz_d, q_d; rewritten only when that changes
  int prepare_inputs();
  InDesc* indesc_d = nullptr;
  InDesc in_user{nullptr, nullptr, 1, 0};  // the caller's device arrays of a pending build
  InDesc in_cur{nullptr, nullptr, 0, 0};   // what indesc_d holds (when in_loaded)
  bool in_pending = false, in_loaded = false;
  OutDesc out_cur{nullptr, nullptr, nullptr, 0, 0};  // what outdesc_d holds
  int field();                    // potentials and fields in one pass (lazily allocated buffers)
  int check_status();
  int delta_energy(int64_t k, const double* x_new, double* de);
  int apply_move(int64_t k, const double* x_new);
  int choose_config(const std::vector<int64_t>& ns) const;
  int choose_side(const std::vector<int64_t>& ns) const;
  int autotune(int reps, int* best, float* best_ms);
  int tune_time_config(int c, int side, int steps, std::vector<float>& t);  // (autotune) steps after a rebuild
  int fail(int code, const char* fmt, ...);
  int cuda_fail(cudaError_t e, const char* what);
  void drop_graphs();

  // configuration
  int device = -1;
  int prec = HSMA_FP32;
  int num_sms = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool use_graphs = true;
  int forced_cfg = -1;
  // where the fused build + potential graph runs the real/Kelvin pair items: 1 = a launch of
  // their own beside the moment chain, 0 = with the surface items after it (issue_fused);
  // forced_side >= 0 forces it, otherwise the tuned choice of the size class or a default
  int forced_side = -1;
  // far field of the real/Kelvin pair sums by the treecode of k_tree.cu (single FP32 system):
  // far_theta = 0 keeps the direct sum; takes effect at the next layout
  double far_theta = 0.0;
  int far_order = 12;
  TreeView tree_view() const;
  cudaEvent_t ev_tree0 = nullptr, ev_tree1 = nullptr;  // around the tree evaluation
  bool tree_timed = false;
  int last_tree_time(float* ms);
  int rk_side = 1;  // the current layout's choice (0, 1 or 2, see issue_fused)
  struct Tuned {
    int bucket, cfg, side;
  };
  std::vector<Tuned> tuned;  // autotuned choices per size class
  std::vector<int> occ_f32, occ_field;
  std::vector<int> regs_f32;  // registers of a CTA of each FP32 pair configuration
  int chain_regs = 0;         // registers of the largest coefficient / surface CTA
  int sm_regs = 65536;        // registers per SM
  int side_ctas_per_sm(int occ) const;
  int occ_f64 = 1, occ_field64 = 1;
  std::vector<SysSpec> spec;

  // layout and workspace
  Layout L;
  std::vector<int64_t> cur_ns;
  bool have_layout = false, layout_uploaded = false;
  char* ws = nullptr;
  size_t ws_cap = 0;
  bool ws_owned = false, ws_user = false;

  // device arrays (carved from the workspace)
  SysDev* sys_d = nullptr;
  double *Mn_d = nullptr, *rec_a_d = nullptr, *rec_b_d = nullptr, *sect_d = nullptr, *inv_np1_d = nullptr;
  float2 *rec_a2_d = nullptr, *rec_b2_d = nullptr, *sect2_d = nullptr;
  float2* mtab_d = nullptr;        // rescaled moment chain: beta_nm, then e_nm sprod_m
  // FP32 path: per-charge moment inputs (k_moment_prep) and the moment units
  float4 *mgeo_d = nullptr, *mz_d = nullptr;
  float2* mwq_d = nullptr;
  double* mcen_d = nullptr;
  int2* itmu_d = nullptr;
  double *xyz_d = nullptr, *q_d = nullptr;
  float4 *srchi_d = nullptr, *srclo_d = nullptr, *surfa_d = nullptr, *surfb_d = nullptr;
  dbl4 *src64_d = nullptr, *surf64a_d = nullptr;
  double* surf64b_d = nullptr;
  float2* part_d = nullptr;
  double* part64_d = nullptr;
  double *mom_d = nullptr, *coef_d = nullptr, *r0_d = nullptr;
  float2* coef2_d = nullptr;      // coefficients as FP32 (hi, lo) pairs
  double* sb_d = nullptr;         // auxiliary-sphere solid-harmonic tables
  int2* itsb_d = nullptr;
  int *perm_d = nullptr, *iperm_d = nullptr;  // spatial order (sorted position <-> input index)
  int* key_d = nullptr;            // cell key of every charge
  int* hist_d = nullptr;           // cell histogram per system, then a sort counter per system (zero
                                   // between builds)
  int* sortscr_d = nullptr;        // scratch of the order's sort (2 ints per charge)
  float4* xs_d = nullptr;          // FP32 path: (hi, lo) split of the inputs (k_order_keys)
  float4* boxes_d = nullptr;      // bounding boxes of 32 consecutive sorted records
  int2* itord_d = nullptr;
  int2* itsort_d = nullptr;
  cudaStream_t side = nullptr;    // second stream of the build (order + records beside the moments)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_img = nullptr;
  int prio_hi = 0, prio_mid = 0;  // greatest stream priority of the device and the next one
                                  // (launch priorities of the overlapped step, issue_fused)
  // deferred build: build() copies the inputs; the first evaluation runs the build, and a
  // potential/energy evaluation runs it fused with the pair sum (overlap) in one graph
  bool build_pending = false;
  bool overlap = true;
  int ensure_built();
  double *phic_d = nullptr, *phir_d = nullptr, *phit_d = nullptr, *epart_d = nullptr, *energy_d = nullptr;
  unsigned int *ctr_pairs_d = nullptr, *ctr_red_d = nullptr, *ctr_delta_d = nullptr;
  int* status_d = nullptr;
  dbl4* surfx_d = nullptr;        // FP64 surface point and weight
  double2* surfqd_d = nullptr;    // FP64 monopole and dipole strength
  double2* vsurf_d = nullptr;     // potentials of the real charges under the two surface kernels
  DeltaReq* dreq_d = nullptr;
  int4* ditems_d = nullptr;
  int2 *dreqit_d = nullptr, *mitems_d = nullptr;
  double *dpart_d = nullptr, *de_d = nullptr;
  int max_requests = 1;           // move requests per launch the layout reserves room for
  bool v_ready = false;
  int ensure_v();
  // batched moves: reqs are (system, k, new position); de receives one double per request
  int delta_batch(const std::vector<DeltaReq>& reqs, double* de_host);
  int move_batch(const std::vector<DeltaReq>& reqs);
  int2 *it12_d = nullptr, *it2r_d = nullptr, *it3_d = nullptr, *it5_d = nullptr, *it3m_d = nullptr;
  int* sel_d = nullptr;
  int2* selrng_d = nullptr;
  int4* it4_d = nullptr;
  int4* it4x_d = nullptr;
  int4* it4f_d = nullptr;
  int4* it4fx_d = nullptr;
  unsigned int* ctr_pairs2_d = nullptr;  // work counter of the overlapped real/Kelvin pair launch

  // pair-kernel timing events (recorded around every pair-sum launch)
  cudaEvent_t ev_pair0 = nullptr, ev_pair1 = nullptr;
  cudaEvent_t ev_pot1 = nullptr;  // after the reduction (pair sum + reduction = potentials pass)
  cudaEvent_t ev_tune0 = nullptr, ev_tune1 = nullptr;  // autotuner: around an overlapped step
  // ordering with the caller's legacy default stream when the handle owns its stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  void enter();
  void leave();
  bool pair_timed = false;
  int last_pair_time(float* ms);
  int last_pot_time(float* ms);

  // state
  bool sources_ready = false, pot_ready = false;
  // energies of the last potential pass staged in pinned host memory by a host-output potential
  // call (batch API), so that an energy call right after it needs no second GPU round trip
  double* energy_h = nullptr;
  size_t energy_h_cap = 0;
  uint64_t pot_epoch = 0, energy_h_epoch = ~uint64_t(0);
  int stage_energies();
  bool energy_parts = false;   // the current energies are per-block terms (epart), not energy_d
  bool energy_h_parts = false; // what the pinned mirror holds
  void energies_from(const double* raw, bool parts, double* out) const;
  int read_energies(double* out);
  // pinned staging of a host-output potential copy and of the status word: one round trip
  char* host_stage = nullptr;
  size_t host_stage_cap = 0;
  int ensure_host_stage(int64_t count);  // call before enqueueing the work whose results are copied
  double* host_stage_dev = nullptr;  // device addresses of the pinned buffers (kernel writes)
  double* energy_h_dev = nullptr;
  // the results of a host-output call: written: the pass just run wrote the values and the
  // energy terms into the pinned buffers itself (OutDesc from host_outputs), else copied here;
  // direct: dst_h is page-locked and was (or is now) written by the device itself
  int copy_to_host(const double* src_d, int64_t count, double* dst_h, bool written = false, bool direct = false);
  OutDesc host_outputs(int64_t count, int what, double* phi_dev = nullptr);
  static int out_lane(int what);  // HSMA_TOTAL / HSMA_REACTION / HSMA_COULOMB -> OutDesc::what
  int decode_status(int st);
  bool field_ready = false;       // E is current when pot_ready && field_ready
  cudaGraphExec_t g_build = nullptr, g_pot = nullptr, g_field = nullptr, g_fused = nullptr, g_field_fused = nullptr;
  // field pass buffers, outside the workspace (allocated on the first field request)
  void* fpart_d = nullptr;        // 32 bytes per (chunk, target) slot
  size_t fpart_cap = 0;
  double* E_d = nullptr;          // E_coul, E_rf, E_total: 3 x (3 totN) doubles
  size_t E_cap = 0;
  double *Ec_d = nullptr, *Er_d = nullptr, *Et_d = nullptr;
  int ensure_field_buffers();
  int64_t launches = 0;
  std::string err;

  Tables tables() const;

 private:
  void carve();
  void issue_moments();  // the moment rows (FP64: k_moments; FP32: k_moment_prep, k_moment_units)
  void issue_build();
  void issue_pot();
  void issue_field();
  void issue_fused();
  void launch_pair_items(PairWork w1, PairWork w2, int grid, cudaStream_t st, bool pdl = false);
  int field_slots() const;
  void launch_field_items(PairWork w1, PairWork w2, int grid, cudaStream_t st, bool pdl = false);
  void launch_field_reduce(cudaStream_t st);
  void issue_field_fused();
  int fused_launch_count() const;
  void issue_tree(cudaStream_t st);
  int tree_launch_count() const;
  int build_launch_count() const;
  int pot_launch_count() const;
  int run_graph(cudaGraphExec_t* g, void (Engine::*issue)());
};

}  // namespace hsma
