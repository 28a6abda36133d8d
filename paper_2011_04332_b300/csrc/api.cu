// C ABI of the npFEM library: cell types, batches and the batched step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/npfem.h"
#include "api_internal.h"
#include "npfem_internal.h"
#include "step_kernel.cuh"
#include "adjoint.cuh"
#include "split_kernels.cuh"
#include "iter_cta.cuh"
#include "contact_kernels.cuh"

using namespace npfem;

namespace {
thread_local std::string g_last_error;

npfem_status fail(npfem_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define NPFEM_CUDA_TRY(expr)                                                              \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? NPFEM_ERR_OOM : NPFEM_ERR_CUDA,       \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                    \
  } while (0)

template <typename D, typename S>
std::vector<D> convert(const std::vector<S>& s) {
  return std::vector<D>(s.begin(), s.end());
}
}  // namespace

struct TypeLaunch {
  int type_index;
  int ncells;
  const int32_t* cell_list;  // device
  int* counter;              // device
  char* scratch;             // owned: slot_bytes per warp slot
  size_t slot_bytes;
  int blocks, warps_per_block, blocks_per_sm;
  int z_in_smem;
  int solve_per_coord;
  size_t smem_bytes;
  char* adj_scratch;         // owned: adjoint workspace (first adjoint call)
  size_t adj_slot;
  // split mode: per-cell workspace and the shapes of k_begin/k_iter and k_solve
  char* cell_scratch;        // owned: cell_slot bytes per cell (first split step)
  size_t cell_slot;
  int it_wpb, it_bps, sv_wpb, sv_bps, sv_smem, sv_percoord, sv_cells;
  // CTA iteration kernels (one cell per CTA, X, U and G in shared memory): warps per cell
  // (0: the one-warp-per-cell kernels) and the CTAs per SM that are resident at that width
  int itc_w = 0, itc_bps = 0;
  int* active = nullptr;  // split mode: [2][ncells] lists of iterating cells (inside cell_scratch)
  int groups = 1;         // split mode: cells split into this many groups with phase-offset chains
  std::vector<int32_t> host_list;  // the type's cells (batch indices, increasing)
};

struct npfem_batch {
  std::vector<const npfem_cell_type*> types;
  std::vector<int32_t> type_of_cell;
  std::vector<int64_t> offsets;
  int64_t n_total = 0;
  int ncells = 0;
  npfem_precision prec = NPFEM_FP64;
  DevAllocs mem;
  const int64_t* d_offsets = nullptr;
  std::vector<TypeLaunch> launches;
  int* d_counters = nullptr;
  unsigned long long* d_phase = nullptr;  // [kPhases] per-phase cycle counters
  bool phase_counting = false;            // kernels add to d_phase only when set
  int sms = 148, smem_optin = 0;
  int mode = 1;  // 0: fused persistent kernel, 1: split kernels (k_begin, k_solve, k_iter)
  // split mode with several cell types: one internal stream per type, forked from and
  // joined back into the caller's stream with events (also under stream capture)
  std::vector<cudaStream_t> type_streams;
  std::vector<cudaEvent_t> type_events;
  cudaEvent_t fork_event = nullptr;
  // solve_streams: the chains' solve launches on streams of their own at the highest
  // priority (the rest of a chain at the lowest), ordered with the chain by two events per
  // chain (to_solve[c]: the chain's work before a solve; from_solve[c]: the solve)
  // solve streams: on in the FP32 form (mixed 10^4 batch -1.9 %, 20 000-cell mix -5.4 % per
  // step), off in the FP64 form, whose iteration kernels are FP64 bound too (+11 %)
  bool solve_streams_on = true;
  std::vector<cudaStream_t> solve_streams;
  std::vector<cudaEvent_t> to_solve, from_solve;
  // optional per-launch kernel timing in split mode: a (start, end) event pair around
  // every launch, per chain (type launch x group) and launch slot (0: k_begin, 1 + 2i:
  // k_solve of iteration i, 2 + 2i: k_iter of iteration i), re-recorded by every step
  bool ktiming = false;
  std::vector<cudaEvent_t> kev;      // [launches.size() * kMaxChains][kTimingSlots][2]
  std::vector<int> k_last_slots;     // slots recorded by the last step, per chain
  std::vector<int> k_last_chains;    // cell type of each chain of the last split step
  cudaEvent_t k_ref = nullptr;       // recorded on the caller's stream at the start of a timed step
  ~npfem_batch() {
    for (cudaEvent_t e : kev) cudaEventDestroy(e);
    if (k_ref) cudaEventDestroy(k_ref);
    for (cudaEvent_t e : pipe_events) cudaEventDestroy(e);
    if (h2d_stream) cudaStreamDestroy(h2d_stream);
    if (d2h_stream) cudaStreamDestroy(d2h_stream);
    for (cudaStream_t s : type_streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : type_events) cudaEventDestroy(e);
    for (cudaStream_t s : solve_streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : to_solve) cudaEventDestroy(e);
    for (cudaEvent_t e : from_solve) cudaEventDestroy(e);
    if (fork_event) cudaEventDestroy(fork_event);
    for (cudaEvent_t e : det_ev)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : stag_events) cudaEventDestroy(e);
    if (roll) cudaFree(roll);
    for (TypeLaunch& L : launches) {
      if (L.scratch) cudaFree(L.scratch);
      if (L.adj_scratch) cudaFree(L.adj_scratch);
      if (L.cell_scratch) cudaFree(L.cell_scratch);
    }
  }
  // pipelined host-buffer steps: copy streams and per-chunk events
  cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
  std::vector<cudaEvent_t> pipe_events;  // [0]: start, [1..kMaxChains]: inputs copied,
                                         // then kMaxChains x launches: chunk done per type, last: outputs copied
  // host-step staging (allocated on first npfem_step_host)
  void* d_x = nullptr;
  void* d_v = nullptr;
  void* d_f = nullptr;
  int32_t* d_iters = nullptr;
  double* d_res = nullptr;
  int32_t* d_status = nullptr;
  int32_t* d_done = nullptr;
  double* d_xstar = nullptr;  // implicit adjoint: the forward step's positions and velocities
  double* d_vstar = nullptr;
  // collisions (npfem_batch_set_collisions): parameters and detection buffers
  bool coll = false;
  bool coll_alloc = false;
  npfem_collision_params coll_p{};
  int64_t coll_T = 0;     // hash-table size (power of two, multiple of the scan block)
  ContactParams cp{};
  cudaEvent_t det_ev[2] = {nullptr, nullptr};  // around the detection kernels (kernel timing on)
  std::vector<cudaEvent_t> stag_events;         // staggered group starts (one per chain)
  bool det_timed = false;                      // the last step recorded det_ev
  // rollout adjoint (npfem_rollout_adjoint): checkpoints, segment states and gradient
  // buffers in one allocation, grown on demand
  char* roll = nullptr;
  size_t roll_bytes = 0;
};

template <typename S>
static void fill_view(npfem_cell_type* t, DevTypeView<S>* v, const S* Dinv, const S* w_tri, const S* c_hinge,
                      const S* K0, const S* w_hinge, const S* mass, const S* inv_mass, const S* inc_coef,
                      const int32_t* tris, const int32_t* hinges, const int32_t* inc_ptr, const int32_t* inc_code,
                      const int32_t* perm, const double* dinv, const int32_t* fcol, const uint32_t* frow,
                      const double* fval, const int32_t* bcol, const uint32_t* brow, const double* bval) {
  const HostType& H = t->host;
  v->n = H.n;
  v->T = H.T;
  v->E = H.E;
  v->nchunks_fwd = (int)H.fwd_meta.size();
  v->nchunks_bwd = (int)H.bwd_meta.size();
  v->tris = tris;
  v->Dinv = Dinv;
  v->w_tri = w_tri;
  v->hinges = hinges;
  v->c_hinge = c_hinge;
  v->K0 = K0;
  v->w_hinge = w_hinge;
  v->mass = mass;
  v->inv_mass = inv_mass;
  v->inc_ptr = inc_ptr;
  v->inc_code = inc_code;
  v->inc_coef = inc_coef;
  v->perm = perm;
  v->dinv = dinv;
  v->fwd_meta = fcol;
  v->fwd_rc = frow;
  v->fwd_val = fval;
  v->bwd_meta = bcol;
  v->bwd_rc = brow;
  v->bwd_val = bval;
  v->A0 = H.A0;
  v->V0 = H.V0;
  v->w_area = H.w_area;
  v->w_vol = H.w_vol;
  v->dt = H.dt;
  v->inv_A0 = 1.0 / H.A0;
  v->inv_V0 = 1.0 / H.V0;
  v->idt2 = 1.0 / (H.dt * H.dt);
  v->inv_dt = 1.0 / H.dt;
  v->inv_n = 1.0 / H.n;
  v->damp_m = H.c_alpha / H.dt;
  v->damp_l = H.c_beta / H.dt;
  v->s_min = H.s_min;
  v->s_max = H.s_max;
  v->limited = (H.s_min != 1.0 || H.s_max != 1.0) ? 1 : 0;
}

template <typename S>
static cudaError_t upload_precision(npfem_cell_type* t, DevTypeView<S>* view, const int32_t* tris, const int32_t* tri4,
                                    const int32_t* hinges, const int32_t* inc_ptr, const int32_t* inc_code,
                                    const int32_t* perm, const double* dinv, const int32_t* fcol,
                                    const uint32_t* frow, const double* fval, const int32_t* bcol,
                                    const uint32_t* brow, const double* bval) {
  const HostType& H = t->host;
  std::vector<double> inv_mass(H.n);
  for (int i = 0; i < H.n; ++i) inv_mass[i] = 1.0 / H.mass[i];
  const S *Dinv, *w_tri, *c_hinge, *K0, *w_hinge, *mass, *im, *coef, *tarea, *hunit;
  cudaError_t e;
  if ((e = t->mem.upload(convert<S>(H.Dinv), &Dinv)) != cudaSuccess) return e;
  if ((e = t->mem.upload(convert<S>(H.w_tri), &w_tri)) != cudaSuccess) return e;
  if ((e = t->mem.upload(convert<S>(H.c_hinge), &c_hinge)) != cudaSuccess) return e;
  if ((e = t->mem.upload(convert<S>(H.K0), &K0)) != cudaSuccess) return e;
  if ((e = t->mem.upload(convert<S>(H.w_hinge), &w_hinge)) != cudaSuccess) return e;
  if ((e = t->mem.upload(convert<S>(H.mass), &mass)) != cudaSuccess) return e;
  if ((e = t->mem.upload(convert<S>(inv_mass), &im)) != cudaSuccess) return e;
  if ((e = t->mem.upload(convert<S>(H.inc_coef), &coef)) != cudaSuccess) return e;
  if ((e = t->mem.upload(convert<S>(H.area), &tarea)) != cudaSuccess) return e;
  if ((e = t->mem.upload(convert<S>(H.hinge_unit), &hunit)) != cudaSuccess) return e;
  view->tri_area = tarea;
  view->hinge_unit = hunit;
  std::vector<double> trc(4 * (size_t)H.T);
  for (int q = 0; q < H.T; ++q) {
    trc[4 * q] = H.Dinv[3 * q];
    trc[4 * q + 1] = H.Dinv[3 * q + 1];
    trc[4 * q + 2] = H.Dinv[3 * q + 2];
    trc[4 * q + 3] = H.w_tri[q];
  }
  const S* trc_d;
  if ((e = t->mem.upload(convert<S>(trc), &trc_d)) != cudaSuccess) return e;
  view->trc = trc_d;
  view->tri4 = tri4;
  fill_view<S>(t, view, Dinv, w_tri, c_hinge, K0, w_hinge, mass, im, coef, tris, hinges, inc_ptr, inc_code, perm,
               dinv, fcol, frow, fval, bcol, brow, bval);
  return cudaSuccess;
}

npfem_status npfem_internal_fail(npfem_status code, const std::string& msg) { return fail(code, msg); }

// Launch shape of one cell type: warps per CTA (1..4), CTAs per SM, and whether each
// warp's FP64 solve vector lives in shared memory.  (Re)allocates the per-warp workspace.
static npfem_status configure_launch(npfem_batch* b, TypeLaunch& L, int wpb, int bps, int zsmem, int per_coord) {
  const HostType& H = b->types[L.type_index]->host;
  if (wpb < 1 || wpb > 4 || bps < 1 || bps > 16) return fail(NPFEM_ERR_INVALID_ARG, "launch: warps/CTA in 1..4, CTAs/SM in 1..16");
  const size_t ssize = b->prec == NPFEM_FP64 ? sizeof(double) : sizeof(float);
  // the per-coordinate sweep only narrows a vector kept in shared memory; a vector in the
  // workspace is always the full [n+1][3] one (the solve sweeps it with the three
  // coordinates together)
  const size_t zbytes = sizeof(double) * (per_coord ? 1 : 3) * ((size_t)H.n + 1);
  const size_t zbytes_ws = sizeof(double) * 3 * ((size_t)H.n + 1);
  const size_t smem = zsmem ? zbytes * wpb : 0;
  if (smem > (size_t)b->smem_optin) return fail(NPFEM_ERR_UNSUPPORTED, "launch: solve vectors exceed shared memory");
  size_t v = (size_t)3 * H.n;
  size_t bytes = ssize * ((8 + 2 * kHistory) * v + 9 * (size_t)H.T + 3 * (size_t)H.E);
  bytes = (bytes + 255) & ~(size_t)255;
  if (!zsmem) bytes += zbytes_ws;
  bytes = (bytes + 255) & ~(size_t)255;
  const int blocks = std::max(1, std::min<int>(b->sms * bps, (L.ncells + wpb - 1) / wpb));
  void* scr = nullptr;
  cudaError_t e = cudaMalloc(&scr, std::max<size_t>(16, bytes * (size_t)blocks * wpb));
  if (e != cudaSuccess) return fail(NPFEM_ERR_OOM, std::string("launch: workspace: ") + cudaGetErrorString(e));
  if (L.scratch) cudaFree(L.scratch);
  if (L.adj_scratch) cudaFree(L.adj_scratch);
  L.scratch = static_cast<char*>(scr);
  L.adj_scratch = nullptr;
  L.adj_slot = 0;
  L.slot_bytes = bytes;
  L.blocks = blocks;
  L.warps_per_block = wpb;
  L.blocks_per_sm = bps;
  L.z_in_smem = zsmem ? 1 : 0;
  L.solve_per_coord = per_coord ? 1 : 0;
  L.smem_bytes = smem;
  return NPFEM_OK;
}

// The solve kernel instantiated for a cell count and vector placement.
template <typename S>
static void (*solve_kernel(int cells, int place))(DevTypeView<S>, StepParams) {
  static void (*const table[4][3])(DevTypeView<S>, StepParams) = {
      {npfem_k_solve<S, 1, kZWorkspace>, npfem_k_solve<S, 1, kZShared>, npfem_k_solve<S, 1, kZSharedPerCoord>},
      {npfem_k_solve<S, 2, kZWorkspace>, npfem_k_solve<S, 2, kZShared>, npfem_k_solve<S, 2, kZSharedPerCoord>},
      {npfem_k_solve<S, 3, kZWorkspace>, npfem_k_solve<S, 3, kZShared>, npfem_k_solve<S, 3, kZSharedPerCoord>},
      {npfem_k_solve<S, 4, kZWorkspace>, npfem_k_solve<S, 4, kZShared>, npfem_k_solve<S, 4, kZSharedPerCoord>}};
  return table[cells - 1][place];
}

// Lets a kernel use up to `optin` bytes of shared memory per block in total (its static
// shared memory included).
template <typename F>
static cudaError_t allow_dynamic_smem(F* kernel, int optin) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)a.sharedSizeBytes);
}

template <typename S>
static cudaError_t set_solve_smem_attr(int bytes) {
  cudaError_t e = cudaSuccess;
  for (int c = 1; c <= 4 && e == cudaSuccess; ++c)
    for (int pl = 1; pl <= 2 && e == cudaSuccess; ++pl) e = allow_dynamic_smem(solve_kernel<S>(c, pl), bytes);
  if (e == cudaSuccess) e = allow_dynamic_smem(npfem_k_solve_cta<S, kCtaWarps[0], 1>, bytes);
  if (e == cudaSuccess) e = allow_dynamic_smem(npfem_k_solve_cta<S, kCtaWarps[1], 1>, bytes);
  if (e == cudaSuccess) e = allow_dynamic_smem(npfem_k_solve_cta<S, kCtaWarps[2], 1>, bytes);
  if (e == cudaSuccess) e = allow_dynamic_smem(npfem_k_solve_cta<S, kCtaWarps[3], 1>, bytes);
  if (e == cudaSuccess) e = allow_dynamic_smem(npfem_k_solve_cta<S, kCtaWarps[0], 2>, bytes);
  if (e == cudaSuccess) e = allow_dynamic_smem(npfem_k_solve_cta<S, kCtaWarps[1], 2>, bytes);
  return e;
}

// Dynamic shared memory of a solve-kernel CTA: per warp, `cells` solve vectors of
// [n+1][3] doubles (or [n+1] per coordinate); placement 2 (the CTA's warps sweep its
// cells together): `cells` vectors of [n+1][3] doubles.
static size_t split_solve_smem(int n, int wpb, int per_coord, int cells, int placement = 1) {
  if (placement == 2) return sizeof(double) * 3 * ((size_t)n + 1) * (size_t)cells;
  return sizeof(double) * (per_coord ? 1 : 3) * ((size_t)n + 1) * (size_t)wpb * (size_t)cells;
}

// Default split-mode shapes by size class, from autotuning on B300 (homogeneous 642-vertex
// batch and the mixed 162/642/2562-vertex batch).
static void default_split_shape(TypeLaunch& L, int n, npfem_precision prec) {
  L.sv_percoord = 0;
  L.sv_cells = 1;
  if (n <= 256) {         // platelet-sized: 14 solve warps/SM, one vector per warp
    L.sv_wpb = 2, L.sv_bps = 7, L.sv_smem = 1;
  } else if (n <= 1024) {  // 642-vertex RBC: CTAs of 2 warps per cell, 13 per SM (72 registers)
    L.sv_wpb = 2, L.sv_bps = 13, L.sv_smem = 2;
  } else {                 // 2562-vertex RBC: CTAs of 8 warps per cell, 3 per SM (80 registers)
    L.sv_wpb = 8, L.sv_bps = 3, L.sv_smem = 2;
  }
  // iteration kernels: 32 warps per SM in the FP32 form (64 registers), 16 in FP64
  L.it_wpb = 2, L.it_bps = prec == NPFEM_FP64 ? 8 : 16;
  // large types run as several concurrent chains that fill each other's wave tails (a
  // batch of one type: see npfem_batch_create)
  L.groups = L.ncells >= 4096 ? 4 : (L.ncells >= 2048 ? 2 : 1);
  // fewer CTAs per SM where the SM cannot hold that many shared vectors; workspace
  // vectors where it cannot hold one
  const size_t cta = split_solve_smem(n, L.sv_wpb, L.sv_percoord, L.sv_cells, L.sv_smem) + 1024;
  while (L.sv_smem && L.sv_bps > 1 && cta * (size_t)L.sv_bps > 228 * 1024) --L.sv_bps;
  if (L.sv_smem && cta > 227 * 1024) {
    L.sv_smem = 0;
    L.sv_wpb = 2, L.sv_bps = 8;
  }
}

// Width of the CTA iteration kernels for an n-vertex type (warps per cell), measured on
// B300 in the FP32 form: 2 warps for platelet-sized cells, 4 for 642 vertices, 8 for 2562
// (the mixed 10^4-cell step: 79.6 ms at 8 warps against 83.2 at 16).  The FP64 form keeps
// the one-warp kernels (0): its objective is bound by the FP64 pipe, not by the gathers
// the shared-memory kernels remove, and the one-warp kernels measured faster (4096-cell
// step 34.5 against 39.5 ms).  The width sets the order of a cell's CTA-wide sums, so it
// is fixed per type unless the caller sets it (npfem_batch_set_iter_width).
static int default_iter_width(int n, npfem_precision prec) {
  if (prec == NPFEM_FP64) return 0;
  return default_cta_warps(n);
}

// Uses the CTA iteration kernels with w warps per cell for the type (w = 0: the warp
// kernels), if the type is coloured and its shared-memory arrays fit a CTA; records the
// resident CTAs per SM at that width.  Returns false if the kernels cannot run the type
// at that width.
static bool set_iter_cta(npfem_batch* b, TypeLaunch& L, int w) {
  L.itc_w = 0;
  L.itc_bps = 0;
  if (w == 0) return true;
  const HostType& H = b->types[L.type_index]->host;
  if (H.tri_cptr.empty() || H.hinge_cptr.empty()) return false;
  const bool f64 = b->prec == NPFEM_FP64;
  const size_t smem = f64 ? iter_cta_smem_bytes<double>(H.n) : iter_cta_smem_bytes<float>(H.n);
  if (smem + sizeof(CtaShared) + 1024 > (size_t)b->smem_optin) return false;  // static shared memory, rounded up
  int nb = 0;
  cudaError_t e = f64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, npfem_k_iter_cta<double, false>, 32 * w, smem)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, npfem_k_iter_cta<float, false>, 32 * w, smem);
  if (e != cudaSuccess || nb < 1) {
    cudaGetLastError();
    return false;
  }
  L.itc_w = w;
  L.itc_bps = nb;
  return true;
}

template <typename S>
static cudaError_t set_iter_cta_smem_attr(int bytes) {
  cudaError_t e = allow_dynamic_smem(npfem_k_begin_cta<S, false>, bytes);
  if (e == cudaSuccess) e = allow_dynamic_smem(npfem_k_begin_cta<S, true>, bytes);
  if (e == cudaSuccess) e = allow_dynamic_smem(npfem_k_iter_cta<S, false>, bytes);
  if (e == cudaSuccess) e = allow_dynamic_smem(npfem_k_iter_cta<S, true>, bytes);
  return e;
}

static npfem_status ensure_cell_scratch(npfem_batch* b, TypeLaunch& L) {
  if (L.cell_scratch) return NPFEM_OK;
  const HostType& H = b->types[L.type_index]->host;
  const size_t ssize = b->prec == NPFEM_FP64 ? sizeof(double) : sizeof(float);
  size_t v = (size_t)3 * H.n;
  size_t bytes = ssize * ((8 + 2 * kHistory) * v + 9 * (size_t)H.T + 3 * (size_t)H.E);
  bytes = (bytes + 255) & ~(size_t)255;
  bytes += sizeof(double) * 3 * ((size_t)H.n + 1);
  bytes = kStateBytes + ((bytes + 255) & ~(size_t)255);
  void* p = nullptr;
  // per-cell slots, then two lists of cell slots (the cells iterating at even / odd iterations)
  cudaError_t e = cudaMalloc(&p, bytes * (size_t)L.ncells + 2 * sizeof(int) * (size_t)L.ncells);
  if (e != cudaSuccess) return fail(NPFEM_ERR_OOM, std::string("split step: workspace: ") + cudaGetErrorString(e));
  L.cell_scratch = static_cast<char*>(p);
  L.cell_slot = bytes;
  L.active = reinterpret_cast<int*>(L.cell_scratch + bytes * (size_t)L.ncells);
  return NPFEM_OK;
}

// One group of a type's cells: list items [g0, g0 + gn) with its own counter block.
struct GroupRange {
  int g0, gn;
  int* counter;
};

template <typename S>
static npfem_status launch_split(npfem_batch* b, const npfem_cell_type* t, const TypeLaunch& L, const GroupRange& G,
                                 StepParams P, int kind, int it, int max_iters, S* x, S* v, const S* f,
                                 const DevTypeView<S>& view, cudaStream_t st) {
  P.ncells_list = G.gn;
  P.cell_list = L.cell_list + G.g0;
  P.scratch = L.cell_scratch + (size_t)G.g0 * L.cell_slot;
  P.slot_bytes = L.cell_slot;
  int* act_count = G.counter + kActiveCountOff;
  int* act0 = L.active + G.g0;                // list of even iterations (item indices of the group)
  int* act1 = L.active + L.ncells + G.g0;     // list of odd iterations
  // CTA iteration kernels: the resident CTAs per SM, capped by the iteration shape's CTAs
  // per SM (fewer leave room on each SM for the solve kernels of other chains)
  const size_t itc_smem = iter_cta_smem_bytes<S>(view.n);
  const int itc_grid = std::max(1, std::min<int>(b->sms * std::min(L.itc_bps, L.it_bps), G.gn));
  if (kind == 0) {
    P.queue_counter = G.counter;
    P.act_out = act0;
    P.act_count_out = act_count;
    int grid = std::max(1, std::min<int>(b->sms * L.it_bps, (G.gn + L.it_wpb - 1) / L.it_wpb));
    if (L.itc_w > 0 && view.limited)
      npfem_k_begin_cta<S, true><<<itc_grid, 32 * L.itc_w, itc_smem, st>>>(view, P, max_iters, x, v, f);
    else if (L.itc_w > 0)
      npfem_k_begin_cta<S, false><<<itc_grid, 32 * L.itc_w, itc_smem, st>>>(view, P, max_iters, x, v, f);
    else if (view.limited)
      npfem_k_begin<S, true><<<grid, 32 * L.it_wpb, 0, st>>>(view, P, max_iters, x, v, f);
    else
      npfem_k_begin<S, false><<<grid, 32 * L.it_wpb, 0, st>>>(view, P, max_iters, x, v, f);
  } else if (kind == 1) {
    P.queue_counter = G.counter + 1 + 2 * it;
    P.act_in = (it & 1) ? act1 : act0;
    P.act_count_in = act_count + it;
    P.z_in_smem = L.sv_smem == 1;
    P.solve_per_coord = L.sv_percoord;
    P.solve_cells = std::max(1, std::min(4, L.sv_cells));
    const HostType& H = t->host;
    if (L.sv_smem == 2 && L.sv_cells == 2) {  // CTA-cooperative, two cells per CTA of sv_wpb warps
      const size_t smem = split_solve_smem(H.n, L.sv_wpb, 0, 2, 2);
      const int grid = std::max(1, std::min<int>(b->sms * L.sv_bps, (G.gn + 1) / 2));
      if (L.sv_wpb == kCtaWarps[0])
        npfem_k_solve_cta<S, kCtaWarps[0], 2><<<grid, 32 * kCtaWarps[0], smem, st>>>(view, P);
      else
        npfem_k_solve_cta<S, kCtaWarps[1], 2><<<grid, 32 * kCtaWarps[1], smem, st>>>(view, P);
    } else if (L.sv_smem == 2) {  // CTA-cooperative: one cell per CTA of sv_wpb warps
      const size_t smem = split_solve_smem(H.n, L.sv_wpb, 0, 1, 2);
      const int grid = std::max(1, std::min<int>(b->sms * L.sv_bps, G.gn));
      switch (L.sv_wpb) {
        case kCtaWarps[0]: npfem_k_solve_cta<S, kCtaWarps[0], 1><<<grid, 32 * kCtaWarps[0], smem, st>>>(view, P); break;
        case kCtaWarps[1]: npfem_k_solve_cta<S, kCtaWarps[1], 1><<<grid, 32 * kCtaWarps[1], smem, st>>>(view, P); break;
        case kCtaWarps[2]: npfem_k_solve_cta<S, kCtaWarps[2], 1><<<grid, 32 * kCtaWarps[2], smem, st>>>(view, P); break;
        default: npfem_k_solve_cta<S, kCtaWarps[3], 1><<<grid, 32 * kCtaWarps[3], smem, st>>>(view, P); break;
      }
    } else {
      size_t smem = L.sv_smem ? split_solve_smem(H.n, L.sv_wpb, L.sv_percoord, P.solve_cells) : 0;
      const int per_cta = L.sv_wpb * P.solve_cells;
      int grid = std::max(1, std::min<int>(b->sms * L.sv_bps, (G.gn + per_cta - 1) / per_cta));
      const int place = !L.sv_smem ? kZWorkspace : (L.sv_percoord ? kZSharedPerCoord : kZShared);
      solve_kernel<S>(P.solve_cells, place)<<<grid, 32 * L.sv_wpb, smem, st>>>(view, P);
    }
  } else {
    P.queue_counter = G.counter + 2 + 2 * it;
    P.act_out = (it & 1) ? act0 : act1;
    P.act_count_out = act_count + it + 1;
    int grid = std::max(1, std::min<int>(b->sms * L.it_bps, (G.gn + L.it_wpb - 1) / L.it_wpb));
    if (L.itc_w > 0 && view.limited)
      npfem_k_iter_cta<S, true><<<itc_grid, 32 * L.itc_w, itc_smem, st>>>(view, P, x, v);
    else if (L.itc_w > 0)
      npfem_k_iter_cta<S, false><<<itc_grid, 32 * L.itc_w, itc_smem, st>>>(view, P, x, v);
    else if (view.limited)
      npfem_k_iter<S, true><<<grid, 32 * L.it_wpb, 0, st>>>(view, P, x, v);
    else
      npfem_k_iter<S, false><<<grid, 32 * L.it_wpb, 0, st>>>(view, P, x, v);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(NPFEM_ERR_CUDA, std::string("split step launch: ") + cudaGetErrorString(e));
  return NPFEM_OK;
}

// Contact detection on the step's input positions (collisions enabled): normals, spatial
// hash, scan, scatter, query; all on stream st, before any step kernel.
template <typename S>
static npfem_status detect_contacts_t(npfem_batch* b, const S* x, cudaStream_t st) {
  ContactParams C = b->cp;
  const int64_t N = b->n_total, T = b->coll_T;
  C.n_total = N;
  C.h = b->coll_p.radius;
  C.h_inv = 1.0 / b->coll_p.radius;
  C.r2 = b->coll_p.radius * b->coll_p.radius;
  C.mask = (uint32_t)(T - 1);
  NPFEM_CUDA_TRY(cudaMemsetAsync(C.count, 0, sizeof(int32_t) * T, st));
  NPFEM_CUDA_TRY(cudaMemsetAsync(C.maxabs, 0, sizeof(int32_t), st));
  for (const TypeLaunch& L : b->launches) {
    const npfem_cell_type* t = b->types[L.type_index];
    const int grid = std::max(1, std::min(b->sms * 16, L.ncells));
    const size_t smem = sizeof(double) * 3 * (size_t)t->host.T;
    if constexpr (sizeof(S) == 8)
      npfem_k_normals<double><<<grid, 128, smem, st>>>(t->v64, L.cell_list, L.ncells, b->d_offsets, N, x, C.nrm);
    else
      npfem_k_normals<float><<<grid, 128, smem, st>>>(t->v32, L.cell_list, L.ncells, b->d_offsets, N, x, C.nrm);
  }
  const int vgrid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)b->sms * 16, (N + 255) / 256));
  npfem_k_hash<S><<<vgrid, 256, 0, st>>>(C, x);
  const int nblk = (int)(T / kScanBlock);
  npfem_k_scan_blocks<<<nblk, kScanThreads, 0, st>>>(C.count, C.start, C.bsum);
  npfem_k_scan_carry<<<1, kScanThreads, 0, st>>>(C.bsum, nblk);
  const int tgrid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)b->sms * 16, (T + 255) / 256));
  npfem_k_scan_add<<<tgrid, 256, 0, st>>>(C, T);
  npfem_k_scatter<S><<<vgrid, 256, 0, st>>>(C, x);
  const int qgrid = (int)std::max<int64_t>(1, (N + 127) / 128);
  npfem_k_query<S><<<qgrid, 128, 0, st>>>(C, x);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(NPFEM_ERR_CUDA, std::string("contact detection: ") + cudaGetErrorString(e));
  return NPFEM_OK;
}

static npfem_status detect_contacts(npfem_batch* b, const void* x, cudaStream_t st) {
  if (b->prec == NPFEM_FP64) return detect_contacts_t<double>(b, static_cast<const double*>(x), st);
  return detect_contacts_t<float>(b, static_cast<const float*>(x), st);
}

// The step kernels' view of the contacts of the current step (null when collisions are off)
// and of the box walls; x is the state being stepped (the cells' anchors are read from it).
static void set_contact_params(const npfem_batch* b, StepParams& P, const void* x) {
  if (!b->coll) return;
  P.contact_count = b->cp.ccount;
  P.contact_plane = b->cp.cplane;
  P.contact_delta = b->coll_p.delta;
  P.contact_weight = b->coll_p.weight;
  P.box = b->coll_p.walls ? b->cp.box : nullptr;
  P.x_state = x;
}

static constexpr int kTimingSlots = 1 + 2 * kSplitMaxIters;

// Records one timing event on stream s; under stream capture it becomes an external
// event-record node of the graph, so graph replays re-record it.
static cudaError_t record_timing_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t err = cudaStreamIsCapturing(s, &cs);
  if (err != cudaSuccess) return err;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
                                             : cudaEventRecord(e, s);
}

// Chunks of a pipelined step: cells [bounds[g], bounds[g+1]) form chunk g; the chains
// of chunk g wait for in[g] and record done[g * ntypes_launched + type launch].
struct PipelinePlan {
  int K;
  const int* bounds;
  cudaEvent_t* in;
  cudaEvent_t* done;
};

// Split-mode step.  Each (type, group) is a chain of kernels -- k_begin, then per
// iteration k_solve and k_iter -- on its own stream when there is more than one chain;
// the chains run concurrently, so they fill each other's wave tails and one chain's
// FP32 iteration kernel overlaps another's FP64 solve.
static npfem_status step_split(npfem_batch* b, void* x, void* v, const void* f_ext, const int32_t* iters,
                               const npfem_solver_opts* opts, int max_iters, double* residual_out,
                               int32_t* status_out, cudaStream_t st, const PipelinePlan* pipe = nullptr) {
  struct Chain {
    size_t li;
    int g;
    GroupRange G;
  };
  std::vector<Chain> chains;
  for (size_t li = 0; li < b->launches.size(); ++li) {
    TypeLaunch& L = b->launches[li];
    npfem_status rc = ensure_cell_scratch(b, L);
    if (rc != NPFEM_OK) return rc;
    if (pipe) {  // chunk g: the type's cells with batch index in [bounds[g], bounds[g+1])
      for (int g = 0; g < pipe->K; ++g) {
        const auto lo = std::lower_bound(L.host_list.begin(), L.host_list.end(), pipe->bounds[g]);
        const auto hi = std::lower_bound(L.host_list.begin(), L.host_list.end(), pipe->bounds[g + 1]);
        const int g0 = (int)(lo - L.host_list.begin()), g1 = (int)(hi - L.host_list.begin());
        chains.push_back({li, g, {g0, g1 - g0, L.counter + (size_t)g * kSplitCounters}});
      }
      continue;
    }
    const int ng = std::max(1, std::min(L.groups, L.ncells));
    for (int g = 0; g < ng; ++g) {
      const int g0 = (int)((int64_t)L.ncells * g / ng), g1 = (int)((int64_t)L.ncells * (g + 1) / ng);
      chains.push_back({li, g, {g0, g1 - g0, L.counter + (size_t)g * kSplitCounters}});
    }
  }
  const size_t nc = chains.size();
  const bool fork = nc > 1;
  if (fork) {
    // Stream priorities: the chains of the type with the most work per step (cells x
    // vertices) run at the highest priority, so the others fill its gaps instead of
    // delaying it.  Streams are (re)created outside stream capture only.
    size_t heavy = 0;
    double most = -1.0;
    for (size_t li = 0; li < b->launches.size(); ++li) {
      const double w = (double)b->launches[li].ncells * b->types[b->launches[li].type_index]->host.n;
      if (w > most) most = w, heavy = li;
    }
    int least = 0, greatest = 0;
    NPFEM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    NPFEM_CUDA_TRY(cudaStreamIsCapturing(st, &cs));
    if (!b->fork_event) NPFEM_CUDA_TRY(cudaEventCreateWithFlags(&b->fork_event, cudaEventDisableTiming));
    for (size_t c = 0; c < nc; ++c) {
      const int want = b->solve_streams_on ? least : (chains[c].li == heavy ? greatest : least);
      if (c < b->type_streams.size()) {
        int have = 0;
        NPFEM_CUDA_TRY(cudaStreamGetPriority(b->type_streams[c], &have));
        if (have == want || cs != cudaStreamCaptureStatusNone) continue;
        NPFEM_CUDA_TRY(cudaStreamSynchronize(b->type_streams[c]));
        NPFEM_CUDA_TRY(cudaStreamDestroy(b->type_streams[c]));
        NPFEM_CUDA_TRY(cudaStreamCreateWithPriority(&b->type_streams[c], cudaStreamNonBlocking, want));
      } else {
        if (cs != cudaStreamCaptureStatusNone)
          return fail(NPFEM_ERR_INVALID_ARG,
                      "split step: first step of this batch configuration under stream capture; run it once uncaptured");
        cudaStream_t s2;
        cudaEvent_t e2;
        NPFEM_CUDA_TRY(cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, want));
        NPFEM_CUDA_TRY(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
        b->type_streams.push_back(s2);
        b->type_events.push_back(e2);
      }
    }
    while (b->solve_streams_on && b->solve_streams.size() < nc) {
      if (cs != cudaStreamCaptureStatusNone)
        return fail(NPFEM_ERR_INVALID_ARG,
                    "split step: first step of this batch configuration under stream capture; run it once uncaptured");
      cudaStream_t s2;
      cudaEvent_t e1, e2;
      NPFEM_CUDA_TRY(cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, greatest));
      NPFEM_CUDA_TRY(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
      NPFEM_CUDA_TRY(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
      b->solve_streams.push_back(s2);
      b->to_solve.push_back(e1);
      b->from_solve.push_back(e2);
    }
  }
  const bool split_solve = fork && b->solve_streams_on;
  if (b->ktiming && b->k_last_slots.size() < nc) {
    return fail(NPFEM_ERR_INVALID_ARG, "split step: kernel timing was enabled for fewer chains; enable it again");
  }
  if (b->ktiming) NPFEM_CUDA_TRY(record_timing_event(b->k_ref, st));
  NPFEM_CUDA_TRY(cudaMemsetAsync(b->d_counters, 0, sizeof(int) * b->types.size() * kMaxChains * kSplitCounters, st));
  if (fork) {
    NPFEM_CUDA_TRY(cudaEventRecord(b->fork_event, st));
    for (size_t c = 0; c < nc; ++c) NPFEM_CUDA_TRY(cudaStreamWaitEvent(b->type_streams[c], b->fork_event, 0));
  }
  StepParams P{};
  P.offsets = b->d_offsets;
  P.n_total = b->n_total;
  P.iters = iters;
  P.iters_default = opts->iters;
  P.residual_out = residual_out;
  P.status_out = status_out;
  P.tol = opts->tol;
  P.iters_done = opts->iters_done;
  P.alpha_log = opts->alpha_log;
  P.alpha_log_len = opts->alpha_log_len;
  P.phase_cycles = b->phase_counting ? b->d_phase : nullptr;
  set_contact_params(b, P, x);
  auto launch = [&](size_t c, int kind, int it, int slot) -> npfem_status {
    const Chain& C = chains[c];
    const TypeLaunch& L = b->launches[C.li];
    const npfem_cell_type* t = b->types[L.type_index];
    cudaStream_t cs = fork ? b->type_streams[c] : st;
    if (split_solve && kind == 1) {  // the solve on the chain's solve stream, after the chain's work
      NPFEM_CUDA_TRY(cudaEventRecord(b->to_solve[c], cs));
      cs = b->solve_streams[c];
      NPFEM_CUDA_TRY(cudaStreamWaitEvent(cs, b->to_solve[c], 0));
    }
    cudaEvent_t* ke = b->ktiming ? &b->kev[(c * kTimingSlots + slot) * 2] : nullptr;
    if (ke) NPFEM_CUDA_TRY(record_timing_event(ke[0], cs));
    npfem_status rc;
    if (b->prec == NPFEM_FP64)
      rc = launch_split<double>(b, t, L, C.G, P, kind, it, max_iters, static_cast<double*>(x),
                                static_cast<double*>(v), static_cast<const double*>(f_ext), t->v64, cs);
    else
      rc = launch_split<float>(b, t, L, C.G, P, kind, it, max_iters, static_cast<float*>(x), static_cast<float*>(v),
                               static_cast<const float*>(f_ext), t->v32, cs);
    if (rc != NPFEM_OK) return rc;
    if (ke) NPFEM_CUDA_TRY(record_timing_event(ke[1], cs));
    if (split_solve && kind == 1) {  // the rest of the chain after the solve
      NPFEM_CUDA_TRY(cudaEventRecord(b->from_solve[c], cs));
      NPFEM_CUDA_TRY(cudaStreamWaitEvent(b->type_streams[c], b->from_solve[c], 0));
    }
    return NPFEM_OK;
  };
  // Staggered groups (one cell type): group g starts when group g-1's k_begin is done, so
  // the groups' FP64 solves and FP32 iteration kernels fall at different times and share
  // the SMs instead of queueing for the same units (4096-cell step 11.23 -> 10.77 ms).  With
  // several types the chains already drift apart; there it measured 1.6 % slower.  The
  // events are created outside stream capture (a captured step after an uncaptured one
  // staggers too; a capture before any step does not).
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  NPFEM_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  const bool stagger = fork && !pipe && b->launches.size() == 1 &&
                       (b->stag_events.size() >= nc || cap == cudaStreamCaptureStatusNone);
  while (stagger && b->stag_events.size() < nc) {
    cudaEvent_t e;
    NPFEM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->stag_events.push_back(e);
  }
  for (size_t c = 0; c < nc; ++c) {
    cudaStream_t cs = fork ? b->type_streams[c] : st;
    if (pipe) NPFEM_CUDA_TRY(cudaStreamWaitEvent(cs, pipe->in[chains[c].g], 0));
    if (chains[c].G.gn == 0) continue;
    if (stagger && c > 0 && chains[c - 1].li == chains[c].li && chains[c - 1].G.gn > 0)
      NPFEM_CUDA_TRY(cudaStreamWaitEvent(cs, b->stag_events[c - 1], 0));
    npfem_status rc = launch(c, 0, 0, 0);
    if (rc != NPFEM_OK) return rc;
    if (stagger) NPFEM_CUDA_TRY(cudaEventRecord(b->stag_events[c], cs));
  }
  for (int it = 0; it < max_iters; ++it) {
    for (size_t c = 0; c < nc; ++c) {
      if (chains[c].G.gn == 0) continue;
      npfem_status rc = launch(c, 1, it, 1 + 2 * it);
      if (rc != NPFEM_OK) return rc;
      rc = launch(c, 2, it, 2 + 2 * it);
      if (rc != NPFEM_OK) return rc;
    }
  }
  if (pipe)
    for (size_t c = 0; c < nc; ++c) {
      cudaStream_t cs = fork ? b->type_streams[c] : st;
      NPFEM_CUDA_TRY(cudaEventRecord(pipe->done[chains[c].g * b->launches.size() + chains[c].li], cs));
    }
  if (b->ktiming)
    for (size_t c = 0; c < nc; ++c) b->k_last_slots[c] = chains[c].G.gn ? 1 + 2 * max_iters : 0;
  b->k_last_chains.assign(nc, 0);
  for (size_t c = 0; c < nc; ++c) b->k_last_chains[c] = b->launches[chains[c].li].type_index;
  if (fork)
    for (size_t c = 0; c < nc; ++c) {
      NPFEM_CUDA_TRY(cudaEventRecord(b->type_events[c], b->type_streams[c]));
      NPFEM_CUDA_TRY(cudaStreamWaitEvent(st, b->type_events[c], 0));
    }
  return NPFEM_OK;
}

extern "C" {

npfem_status npfem_last_error_string(char* buf, size_t len) {
  if (!buf || len == 0) return NPFEM_ERR_INVALID_ARG;
  std::snprintf(buf, len, "%s", g_last_error.c_str());
  return NPFEM_OK;
}

// Strain limits of a material: both 0 means the rotations [1, 1]; otherwise
// 0 < s_min <= 1 <= s_max < inf.
static bool strain_limits(const npfem_material* mat, double* lo, double* hi) {
  if (mat->s_min == 0.0 && mat->s_max == 0.0) {
    *lo = *hi = 1.0;
    return true;
  }
  *lo = mat->s_min;
  *hi = mat->s_max;
  return *lo > 0.0 && *lo <= 1.0 && *hi >= 1.0 && std::isfinite(*hi);
}

npfem_status npfem_create_cell_type(const npfem_mesh* mesh, const npfem_material* mat, double dt,
                                    npfem_cell_type** out) {
  if (!mesh || !mat || !out) return fail(NPFEM_ERR_INVALID_ARG, "create_cell_type: null argument");
  *out = nullptr;
  double s_lo, s_hi;
  if (!strain_limits(mat, &s_lo, &s_hi))
    return fail(NPFEM_ERR_INVALID_ARG, "create_cell_type: strain limits must be 0 < s_min <= 1 <= s_max (finite), "
                                       "or both 0");
  auto* t = new (std::nothrow) npfem_cell_type();
  if (!t) return fail(NPFEM_ERR_OOM, "create_cell_type: host allocation failed");
  std::string err;
  int rc = build_host_type(mesh->n_verts, mesh->n_tris, mesh->rest_xyz, mesh->tris, mat->w_strain, mat->w_bend,
                           mat->w_area, mat->w_vol, mat->density, dt, mat->c_alpha, mat->c_beta, &t->host, &err);
  if (rc != NPFEM_OK) {
    delete t;
    return fail(rc, err);
  }
  t->host.s_min = s_lo;
  t->host.s_max = s_hi;
  cudaError_t e = cudaGetDevice(&t->device);
  const HostType& H = t->host;
  const int32_t *tris, *tri4, *hinges, *inc_ptr, *inc_code, *perm, *fcol, *bcol, *tcp, *hcp;
  std::vector<int32_t> tri4_h(4 * (size_t)H.T, 0);
  for (int q = 0; q < H.T; ++q)
    for (int k = 0; k < 3; ++k) tri4_h[4 * q + k] = H.tris[3 * q + k];
  const uint32_t *frow, *brow;
  const double *dinv, *fval, *bval;
#define UP(vec, ptr)                                      \
  if (e == cudaSuccess) e = t->mem.upload(vec, &ptr);
  UP(H.tris, tris);
  UP(tri4_h, tri4);
  UP(H.hinges, hinges);
  UP(H.inc_ptr, inc_ptr);
  UP(H.inc_code, inc_code);
  UP(H.perm, perm);
  UP(H.dinv, dinv);
  UP(H.fwd_meta, fcol);
  UP(H.fwd_rc, frow);
  UP(H.fwd_val, fval);
  UP(H.bwd_meta, bcol);
  UP(H.bwd_rc, brow);
  UP(H.bwd_val, bval);
  UP(H.tri_cptr, tcp);
  UP(H.hinge_cptr, hcp);
#undef UP
  const int32_t *cfm[kCtaPacks], *cbm[kCtaPacks];
  const uint32_t *cfr[kCtaPacks], *cbr[kCtaPacks];
  const double *cfv[kCtaPacks], *cbv[kCtaPacks];
  for (int i = 0; i < kCtaPacks; ++i) {
    const HostType::LevelPack& P = H.cta[i];
    if (e == cudaSuccess) e = t->mem.upload(P.fwd_meta, &cfm[i]);
    if (e == cudaSuccess) e = t->mem.upload(P.fwd_rc, &cfr[i]);
    if (e == cudaSuccess) e = t->mem.upload(P.fwd_val, &cfv[i]);
    if (e == cudaSuccess) e = t->mem.upload(P.bwd_meta, &cbm[i]);
    if (e == cudaSuccess) e = t->mem.upload(P.bwd_rc, &cbr[i]);
    if (e == cudaSuccess) e = t->mem.upload(P.bwd_val, &cbv[i]);
  }
  if (e == cudaSuccess)
    e = upload_precision<double>(t, &t->v64, tris, tri4, hinges, inc_ptr, inc_code, perm, dinv, fcol, frow, fval, bcol,
                                 brow, bval);
  if (e == cudaSuccess)
    e = upload_precision<float>(t, &t->v32, tris, tri4, hinges, inc_ptr, inc_code, perm, dinv, fcol, frow, fval, bcol,
                                brow, bval);
  if (e == cudaSuccess) {
    const int ntc = H.tri_cptr.empty() ? 0 : (int)H.tri_cptr.size() - 1;
    const int nhc = H.hinge_cptr.empty() ? 0 : (int)H.hinge_cptr.size() - 1;
    t->v64.ntc = t->v32.ntc = ntc;
    t->v64.nhc = t->v32.nhc = nhc;
    t->v64.tri_cptr = t->v32.tri_cptr = tcp;
    t->v64.hinge_cptr = t->v32.hinge_cptr = hcp;
    for (int i = 0; i < kCtaPacks; ++i) {
      const HostType::LevelPack& P = H.cta[i];
      const int nf = (int)P.fwd_meta.size() / P.W, nb = (int)P.bwd_meta.size() / P.W;
      t->v64.cta_nlev_fwd[i] = t->v32.cta_nlev_fwd[i] = nf;
      t->v64.cta_nlev_bwd[i] = t->v32.cta_nlev_bwd[i] = nb;
      t->v64.cta_fwd_meta[i] = t->v32.cta_fwd_meta[i] = cfm[i];
      t->v64.cta_fwd_rc[i] = t->v32.cta_fwd_rc[i] = cfr[i];
      t->v64.cta_fwd_val[i] = t->v32.cta_fwd_val[i] = cfv[i];
      t->v64.cta_bwd_meta[i] = t->v32.cta_bwd_meta[i] = cbm[i];
      t->v64.cta_bwd_rc[i] = t->v32.cta_bwd_rc[i] = cbr[i];
      t->v64.cta_bwd_val[i] = t->v32.cta_bwd_val[i] = cbv[i];
    }
  }
  if (e != cudaSuccess) {
    delete t;
    return fail(e == cudaErrorMemoryAllocation ? NPFEM_ERR_OOM : NPFEM_ERR_CUDA,
                std::string("create_cell_type: device upload failed: ") + cudaGetErrorString(e));
  }
  *out = t;
  return NPFEM_OK;
}

npfem_status npfem_destroy_cell_type(npfem_cell_type* type) {
  if (!type) return fail(NPFEM_ERR_INVALID_ARG, "destroy_cell_type: null");
  delete type;
  return NPFEM_OK;
}

npfem_status npfem_cell_type_info(const npfem_cell_type* t, npfem_type_info* info) {
  if (!t || !info) return fail(NPFEM_ERR_INVALID_ARG, "cell_type_info: null argument");
  const HostType& H = t->host;
  info->n_verts = H.n;
  info->n_tris = H.T;
  info->n_hinges = H.E;
  info->nnz_factor = H.nnz_factor;
  info->solve_chunks = (int64_t)H.fwd_meta.size();
  info->rest_area = H.A0;
  info->rest_volume = H.V0;
  info->total_mass = H.total_mass;
  info->tri_colours = H.tri_cptr.empty() ? 0 : (int32_t)H.tri_cptr.size() - 1;
  info->hinge_colours = H.hinge_cptr.empty() ? 0 : (int32_t)H.hinge_cptr.size() - 1;
  return NPFEM_OK;
}

npfem_status npfem_cell_type_analyze(const npfem_mesh* mesh, const npfem_material* mat, double dt,
                                     npfem_type_info* info) {
  if (!mesh || !mat || !info) return fail(NPFEM_ERR_INVALID_ARG, "cell_type_analyze: null argument");
  double s_lo, s_hi;
  if (!strain_limits(mat, &s_lo, &s_hi))
    return fail(NPFEM_ERR_INVALID_ARG, "cell_type_analyze: strain limits must be 0 < s_min <= 1 <= s_max (finite), "
                                       "or both 0");
  HostType H;
  std::string err;
  int rc = build_host_type(mesh->n_verts, mesh->n_tris, mesh->rest_xyz, mesh->tris, mat->w_strain, mat->w_bend,
                           mat->w_area, mat->w_vol, mat->density, dt, mat->c_alpha, mat->c_beta, &H, &err);
  if (rc != NPFEM_OK) return fail(rc, err);
  info->n_verts = H.n;
  info->n_tris = H.T;
  info->n_hinges = H.E;
  info->nnz_factor = H.nnz_factor;
  info->solve_chunks = (int64_t)H.fwd_meta.size();
  info->rest_area = H.A0;
  info->rest_volume = H.V0;
  info->total_mass = H.total_mass;
  info->tri_colours = H.tri_cptr.empty() ? 0 : (int32_t)H.tri_cptr.size() - 1;
  info->hinge_colours = H.hinge_cptr.empty() ? 0 : (int32_t)H.hinge_cptr.size() - 1;
  return NPFEM_OK;
}

npfem_status npfem_batch_create(const npfem_cell_type* const* types, int32_t ntypes, const int32_t* type_of_cell,
                                int32_t ncells, npfem_precision prec, npfem_batch** out) {
  if (!out || !types || ntypes <= 0 || ncells < 0 || (ncells > 0 && !type_of_cell))
    return fail(NPFEM_ERR_INVALID_ARG, "batch_create: bad arguments");
  if (prec != NPFEM_FP64 && prec != NPFEM_FP32FORM) return fail(NPFEM_ERR_INVALID_ARG, "batch_create: bad precision");
  *out = nullptr;
  for (int i = 0; i < ntypes; ++i)
    if (!types[i]) return fail(NPFEM_ERR_INVALID_ARG, "batch_create: null type");
  for (int c = 0; c < ncells; ++c)
    if (type_of_cell[c] < 0 || type_of_cell[c] >= ntypes)
      return fail(NPFEM_ERR_INVALID_ARG, "batch_create: type_of_cell out of range");
  auto* b = new (std::nothrow) npfem_batch();
  if (!b) return fail(NPFEM_ERR_OOM, "batch_create: host allocation failed");
  b->types.assign(types, types + ntypes);
  b->type_of_cell.assign(type_of_cell, type_of_cell + ncells);
  b->ncells = ncells;
  b->prec = prec;
  b->solve_streams_on = prec != NPFEM_FP64;
  b->offsets.assign(ncells + 1, 0);
  for (int c = 0; c < ncells; ++c) b->offsets[c + 1] = b->offsets[c] + types[type_of_cell[c]]->host.n;
  b->n_total = b->offsets[ncells];
  auto cleanup = [&](npfem_status code, const std::string& msg) {
    delete b;
    return fail(code, msg);
  };
  cudaError_t e = b->mem.upload(b->offsets, &b->d_offsets);
  if (e != cudaSuccess) return cleanup(NPFEM_ERR_CUDA, std::string("batch_create: ") + cudaGetErrorString(e));
  void* cnt = nullptr;
  e = b->mem.alloc(sizeof(int) * ntypes * kMaxChains * kSplitCounters, &cnt);
  if (e != cudaSuccess) return cleanup(NPFEM_ERR_OOM, std::string("batch_create: ") + cudaGetErrorString(e));
  b->d_counters = static_cast<int*>(cnt);
  void* ph = nullptr;
  e = b->mem.alloc(sizeof(unsigned long long) * kPhases, &ph);
  if (e != cudaSuccess) return cleanup(NPFEM_ERR_OOM, std::string("batch_create: ") + cudaGetErrorString(e));
  b->d_phase = static_cast<unsigned long long*>(ph);
  e = cudaMemset(ph, 0, sizeof(unsigned long long) * kPhases);
  if (e != cudaSuccess) return cleanup(NPFEM_ERR_CUDA, std::string("batch_create: ") + cudaGetErrorString(e));
  int dev = 0, sms = 148, smem_optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  b->sms = sms;
  b->smem_optin = smem_optin;
  e = cudaFuncSetAttribute(npfem_step_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(npfem_step_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
  if (e == cudaSuccess) e = allow_dynamic_smem(npfem_adjoint_kernel, smem_optin);
  if (e == cudaSuccess) e = allow_dynamic_smem(npfem_adjoint_implicit_kernel, smem_optin);
  if (e == cudaSuccess)
    e = set_solve_smem_attr<double>(smem_optin);
  if (e == cudaSuccess)
    e = set_solve_smem_attr<float>(smem_optin);
  if (e == cudaSuccess) e = set_iter_cta_smem_attr<double>(smem_optin);
  if (e == cudaSuccess) e = set_iter_cta_smem_attr<float>(smem_optin);
  if (e != cudaSuccess) return cleanup(NPFEM_ERR_CUDA, std::string("batch_create: ") + cudaGetErrorString(e));
  const size_t ssize = prec == NPFEM_FP64 ? sizeof(double) : sizeof(float);
  for (int ti = 0; ti < ntypes; ++ti) {
    std::vector<int32_t> list;
    for (int c = 0; c < ncells; ++c)
      if (type_of_cell[c] == ti) list.push_back(c);
    if (list.empty()) continue;
    const HostType& H = types[ti]->host;
    TypeLaunch L{};
    L.type_index = ti;
    L.ncells = (int)list.size();
    const int32_t* dl = nullptr;
    if ((e = b->mem.upload(list, &dl)) != cudaSuccess)
      return cleanup(NPFEM_ERR_OOM, std::string("batch_create: ") + cudaGetErrorString(e));
    L.cell_list = dl;
    L.host_list = list;
    L.counter = b->d_counters + (size_t)ti * kMaxChains * kSplitCounters;  // chain 0's block
    // default shape: 4 warps per CTA and 3 CTAs per SM, solve vectors in shared memory
    // when four of them fit in 72 KB (n <= 767), else in the workspace
    const size_t zbytes = sizeof(double) * 3 * ((size_t)H.n + 1);
    const int zs = zbytes * 4 <= 72 * 1024 ? 1 : 0;
    default_split_shape(L, H.n, prec);
    set_iter_cta(b, L, default_iter_width(H.n, prec));  // else the warp kernels
    npfem_status rc = configure_launch(b, L, 4, 3, zs, 0);
    if (rc != NPFEM_OK) {
      for (TypeLaunch& P : b->launches) {
        if (P.scratch) cudaFree(P.scratch);
        P.scratch = nullptr;
      }
      if (L.scratch) cudaFree(L.scratch);
      std::string msg = g_last_error;
      delete b;
      return fail(rc, msg);
    }
    b->launches.push_back(L);
  }
  // A batch of one cell type has no other type's chains to overlap with: in the FP32
  // form its groups are its only concurrency, so it splits from 512 cells on (4 groups
  // from 1024).  With several types each type keeps the rule of default_split_shape (more
  // groups measured slower there: their chains already overlap), and so does the FP64
  // form, whose iteration kernels compete with the solves for the FP64 pipe (1024 cells:
  // 4 groups measured 16 % slower than 1).
  if (b->launches.size() == 1 && prec != NPFEM_FP64) {
    TypeLaunch& L = b->launches[0];
    L.groups = L.ncells >= 1024 ? 4 : (L.ncells >= 512 ? 2 : 1);
  }
  *out = b;
  return NPFEM_OK;
}

npfem_status npfem_batch_destroy(npfem_batch* batch) {
  if (!batch) return fail(NPFEM_ERR_INVALID_ARG, "batch_destroy: null");
  delete batch;
  return NPFEM_OK;
}

npfem_status npfem_batch_layout(const npfem_batch* b, int64_t* n_total, int64_t* offsets) {
  if (!b) return fail(NPFEM_ERR_INVALID_ARG, "batch_layout: null batch");
  if (n_total) *n_total = b->n_total;
  if (offsets) std::memcpy(offsets, b->offsets.data(), sizeof(int64_t) * b->offsets.size());
  return NPFEM_OK;
}

npfem_status npfem_step(npfem_batch* b, void* x, void* v, const void* f_ext, const int32_t* iters,
                        const npfem_solver_opts* opts, double* residual_out, int32_t* status_out, void* stream) {
  if (!b || !opts) return fail(NPFEM_ERR_INVALID_ARG, "step: null batch or opts");
  if (b->ncells == 0) return NPFEM_OK;
  if (!x || !v || !f_ext) return fail(NPFEM_ERR_INVALID_ARG, "step: null state array");
  if (opts->iters < 0) return fail(NPFEM_ERR_INVALID_ARG, "step: negative iteration count");
  if (opts->alpha_log_len < 0 || (opts->alpha_log_len > 0 && !opts->alpha_log))
    return fail(NPFEM_ERR_INVALID_ARG, "step: bad alpha log");
  if (!(opts->tol >= 0.0) || std::isinf(opts->tol))
    return fail(NPFEM_ERR_INVALID_ARG, "step: tol must be finite and >= 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  b->det_timed = false;
  if (b->coll) {
    const bool timed = b->ktiming && b->det_ev[0] && b->det_ev[1];
    if (timed) NPFEM_CUDA_TRY(record_timing_event(b->det_ev[0], st));
    npfem_status rc = detect_contacts(b, x, st);
    if (rc != NPFEM_OK) return rc;
    if (timed) NPFEM_CUDA_TRY(record_timing_event(b->det_ev[1], st));
    b->det_timed = timed;
  }
  if (b->mode == 1 && (iters == nullptr || opts->max_iters > 0)) {
    const int max_iters = iters ? opts->max_iters : opts->iters;
    if (max_iters <= kSplitMaxIters) return step_split(b, x, v, f_ext, iters, opts, max_iters, residual_out, status_out, st);
  }
  NPFEM_CUDA_TRY(cudaMemsetAsync(b->d_counters, 0, sizeof(int) * b->types.size() * kMaxChains * kSplitCounters, st));
  for (const TypeLaunch& L : b->launches) {
    const npfem_cell_type* t = b->types[L.type_index];
    StepParams P{};
    P.ncells_list = L.ncells;
    P.cell_list = L.cell_list;
    P.offsets = b->d_offsets;
    P.n_total = b->n_total;
    P.iters = iters;
    P.iters_default = opts->iters;
    P.residual_out = residual_out;
    P.status_out = status_out;
    P.tol = opts->tol;
    P.iters_done = opts->iters_done;
    P.alpha_log = opts->alpha_log;
    P.alpha_log_len = opts->alpha_log_len;
    P.queue_counter = L.counter;
    P.scratch = L.scratch;
    P.slot_bytes = L.slot_bytes;
    P.z_in_smem = L.z_in_smem;
    P.solve_per_coord = L.solve_per_coord;
    P.phase_cycles = b->phase_counting ? b->d_phase : nullptr;
    set_contact_params(b, P, x);
    dim3 grid(L.blocks), block(32 * L.warps_per_block);
    if (b->prec == NPFEM_FP64)
      npfem_step_kernel<double><<<grid, block, L.smem_bytes, st>>>(t->v64, P, static_cast<double*>(x),
                                                                   static_cast<double*>(v),
                                                                   static_cast<const double*>(f_ext));
    else
      npfem_step_kernel<float><<<grid, block, L.smem_bytes, st>>>(t->v32, P, static_cast<float*>(x),
                                                                  static_cast<float*>(v),
                                                                  static_cast<const float*>(f_ext));
    NPFEM_CUDA_TRY(cudaGetLastError());
  }
  return NPFEM_OK;
}

// The adjoint workspace of every type (first adjoint call): per warp slot of the fused
// launch, the unrolled adjoint's tape and vectors (the implicit adjoint uses six of them).
static npfem_status ensure_adjoint_workspace(npfem_batch* b) {
  for (TypeLaunch& L : b->launches) {
    if (L.adj_scratch) continue;
    const HostType& H = b->types[L.type_index]->host;
    size_t v3 = (size_t)3 * H.n;
    size_t nvec = 3 * (size_t)(kMaxAdjIters + 1) + 4 * (size_t)kMaxAdjIters + 2 * (size_t)(kHistory + 1) + 6;
    nvec = std::max<size_t>(nvec, kImplicitVectors);
    size_t bytes = ((sizeof(double) * (nvec * v3 + 3 * kMaxAdjIters) + sizeof(int) * kMaxAdjIters) + 255) &
                   ~(size_t)255;
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes * (size_t)L.blocks * L.warps_per_block);
    if (e != cudaSuccess) return fail(NPFEM_ERR_OOM, std::string("adjoint workspace: ") + cudaGetErrorString(e));
    L.adj_scratch = static_cast<char*>(p);
    L.adj_slot = bytes;
  }
  return NPFEM_OK;
}

npfem_status npfem_step_adjoint(npfem_batch* b, const void* x, const void* v, const void* f_ext,
                                const int32_t* iters, const npfem_solver_opts* opts, const double* gx_next,
                                const double* gv_next, double* gx, double* gv, double* gf, double* gw,
                                int32_t* status_out, void* stream) {
  if (!b || !opts) return fail(NPFEM_ERR_INVALID_ARG, "step_adjoint: null batch or opts");
  if (b->prec != NPFEM_FP64) return fail(NPFEM_ERR_INVALID_ARG, "step_adjoint: needs an FP64 batch");
  if (b->ncells == 0) return NPFEM_OK;
  if (!x || !v || !f_ext || !gx_next || !gx || !gv || !gf || !gw)
    return fail(NPFEM_ERR_INVALID_ARG, "step_adjoint: null array");
  if (opts->iters < 0 || opts->iters > kMaxAdjIters)
    return fail(NPFEM_ERR_INVALID_ARG, "step_adjoint: iteration count must be in [0, 16]");
  if (opts->tol != 0.0)
    return fail(NPFEM_ERR_INVALID_ARG, "step_adjoint: tol must be 0 (fixed iteration counts)");
  if (b->coll)
    return fail(NPFEM_ERR_INVALID_ARG, "step_adjoint: collisions are enabled (contacts are not differentiated)");

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  npfem_status arc = ensure_adjoint_workspace(b);
  if (arc != NPFEM_OK) return arc;
  NPFEM_CUDA_TRY(cudaMemsetAsync(b->d_counters, 0, sizeof(int) * b->types.size() * kMaxChains * kSplitCounters, st));
  for (size_t li = 0; li < b->launches.size(); ++li) {
    const TypeLaunch& L = b->launches[li];
    const npfem_cell_type* t = b->types[L.type_index];
    StepParams P{};
    P.ncells_list = L.ncells;
    P.cell_list = L.cell_list;
    P.offsets = b->d_offsets;
    P.n_total = b->n_total;
    P.iters = iters;
    P.iters_default = opts->iters;
    P.residual_out = nullptr;
    P.status_out = status_out;
    P.alpha_log = nullptr;
    P.alpha_log_len = 0;
    P.queue_counter = L.counter;
    P.scratch = L.scratch;
    P.slot_bytes = L.slot_bytes;
    P.z_in_smem = L.z_in_smem;
    P.solve_per_coord = L.solve_per_coord;
    P.phase_cycles = b->phase_counting ? b->d_phase : nullptr;
    AdjParams A;
    A.gx_next = gx_next;
    A.gv_next = gv_next;
    A.gx = gx;
    A.gv = gv;
    A.gf = gf;
    A.gw = gw;
    A.scratch = L.adj_scratch;
    A.slot_bytes = L.adj_slot;
    const HostType& H = t->host;
    A.w_mat[0] = 0;
    A.w_mat[1] = 0;
    A.w_mat[2] = H.w_area;
    A.w_mat[3] = H.w_vol;
    // one CTA of kAdjWarps warps per cell, over the launch's warp slots (one slot and one
    // solve vector in shared memory per CTA)
    const int adj_blocks = std::max(1, std::min(L.blocks * L.warps_per_block, L.ncells));
    npfem_adjoint_kernel<<<adj_blocks, 32 * kAdjWarps, L.smem_bytes / L.warps_per_block, st>>>(
        t->v64, P, A, static_cast<const double*>(x), static_cast<const double*>(v), static_cast<const double*>(f_ext));
    NPFEM_CUDA_TRY(cudaGetLastError());
  }
  return NPFEM_OK;
}

}  // extern "C"

// Rollout adjoint helpers: y += x; a |= c; out4 += sum over the listed cells of gw[c][0..3]
// in a fixed order (one CTA per cell type, strided per-thread sums, then a tree in shared
// memory), so the per-type weight gradients are bit-for-bit reproducible.
__global__ void npfem_k_add(double* __restrict__ y, const double* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}
__global__ void npfem_k_or(int32_t* __restrict__ a, const int32_t* __restrict__ c, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] |= c[i];
}
constexpr int kTypeSumThreads = 256;
__global__ void __launch_bounds__(kTypeSumThreads) npfem_k_type_sum(const double* __restrict__ gw,
                                                                     const int32_t* __restrict__ cells, int ncells,
                                                                     double* __restrict__ out4) {
  __shared__ double red[4][kTypeSumThreads];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < ncells; i += kTypeSumThreads)
    for (int q = 0; q < 4; ++q) acc[q] += gw[4 * (size_t)cells[i] + q];
  for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = kTypeSumThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out4[threadIdx.x] += red[threadIdx.x][0];
}

static int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 148 * 16)); }

extern "C" {

npfem_status npfem_rollout_adjoint(npfem_batch* b, const double* x0, const double* v0, const double* f_ext,
                                   const int32_t* iters, const npfem_solver_opts* opts, int32_t nsteps,
                                   int32_t ckpt_every, const double* gx_end, const double* gv_end, double* gx0,
                                   double* gv0, double* gf, double* gweights, int32_t* status_out, void* stream) {
  if (!b || !opts) return fail(NPFEM_ERR_INVALID_ARG, "rollout_adjoint: null batch or opts");
  if (b->prec != NPFEM_FP64) return fail(NPFEM_ERR_INVALID_ARG, "rollout_adjoint: needs an FP64 batch");
  if (nsteps < 1 || ckpt_every < 1)
    return fail(NPFEM_ERR_INVALID_ARG, "rollout_adjoint: nsteps and ckpt_every must be >= 1");
  if (!gweights) return fail(NPFEM_ERR_INVALID_ARG, "rollout_adjoint: null gweights");
  if (opts->tol != 0.0)
    return fail(NPFEM_ERR_INVALID_ARG, "rollout_adjoint: tol must be 0 (fixed iteration counts)");
  if (b->coll)
    return fail(NPFEM_ERR_INVALID_ARG, "rollout_adjoint: collisions are enabled (contacts are not differentiated)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t ntypes = b->types.size();
  NPFEM_CUDA_TRY(cudaMemsetAsync(gweights, 0, sizeof(double) * 4 * ntypes, st));
  if (b->ncells == 0) return NPFEM_OK;
  if (!x0 || !v0 || !f_ext || !gx_end || !gx0 || !gv0 || !gf)
    return fail(NPFEM_ERR_INVALID_ARG, "rollout_adjoint: null array");
  if (opts->iters < 0 || opts->iters > kMaxAdjIters)
    return fail(NPFEM_ERR_INVALID_ARG, "rollout_adjoint: iteration count must be in [0, 16]");
  // workspace: ncp checkpoints and K segment states of (x, v), the running state, two
  // (gx, gv) pairs, one step's gf, per-cell gw and statuses
  const int K = ckpt_every, ncp = (nsteps + K - 1) / K;
  const size_t nv = (size_t)3 * b->n_total, vb = sizeof(double) * nv;
  const size_t need = vb * (2 * (size_t)ncp + 2 * (size_t)K + 2 + 4 + 1) + sizeof(double) * 4 * (size_t)b->ncells +
                      sizeof(int32_t) * (size_t)b->ncells + 256;
  if (need > b->roll_bytes) {
    if (b->roll) {
      NPFEM_CUDA_TRY(cudaStreamSynchronize(st));
      cudaFree(b->roll);
      b->roll = nullptr;
      b->roll_bytes = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, need);
    if (e != cudaSuccess) return fail(NPFEM_ERR_OOM, std::string("rollout_adjoint: workspace: ") + cudaGetErrorString(e));
    b->roll = static_cast<char*>(p);
    b->roll_bytes = need;
  }
  double* base = reinterpret_cast<double*>(b->roll);
  double* ck = base;                                  // [ncp][2][3N]
  double* seg = ck + 2 * (size_t)ncp * nv;            // [K][2][3N]
  double* xw = seg + 2 * (size_t)K * nv;              // running x, v
  double* vw = xw + nv;
  double* g[4] = {vw + nv, vw + 2 * nv, vw + 3 * nv, vw + 4 * nv};  // (gx, gv) pairs a and b
  double* gfs = vw + 5 * nv;
  double* gwc = gfs + nv;                             // [ncells][4]
  int32_t* sts = reinterpret_cast<int32_t*>(gwc + 4 * (size_t)b->ncells);
  const int32_t* ssrc = status_out ? sts : nullptr;
  if (status_out) NPFEM_CUDA_TRY(cudaMemsetAsync(status_out, 0, sizeof(int32_t) * b->ncells, st));
  npfem_solver_opts fo = *opts;
  fo.alpha_log = nullptr;
  fo.alpha_log_len = 0;
  fo.iters_done = nullptr;
  auto step_fwd = [&](double* x, double* v) -> npfem_status {
    npfem_status rc = npfem_step(b, x, v, f_ext, iters, &fo, nullptr, status_out ? sts : nullptr, stream);
    if (rc == NPFEM_OK && status_out) npfem_k_or<<<grid_for(b->ncells), 256, 0, st>>>(status_out, ssrc, b->ncells);
    return rc;
  };
  // forward: checkpoint (x, v) before steps 0, K, 2K, ...
  NPFEM_CUDA_TRY(cudaMemcpyAsync(xw, x0, vb, cudaMemcpyDeviceToDevice, st));
  NPFEM_CUDA_TRY(cudaMemcpyAsync(vw, v0, vb, cudaMemcpyDeviceToDevice, st));
  for (int s = 0; s < nsteps; ++s) {
    if (s % K == 0) {
      NPFEM_CUDA_TRY(cudaMemcpyAsync(ck + 2 * (size_t)(s / K) * nv, xw, vb, cudaMemcpyDeviceToDevice, st));
      NPFEM_CUDA_TRY(cudaMemcpyAsync(ck + (2 * (size_t)(s / K) + 1) * nv, vw, vb, cudaMemcpyDeviceToDevice, st));
    }
    npfem_status rc = step_fwd(xw, vw);
    if (rc != NPFEM_OK) return rc;
  }
  // reverse: per segment, recompute its states from the checkpoint, then the step adjoints
  NPFEM_CUDA_TRY(cudaMemcpyAsync(g[0], gx_end, vb, cudaMemcpyDeviceToDevice, st));
  if (gv_end)
    NPFEM_CUDA_TRY(cudaMemcpyAsync(g[1], gv_end, vb, cudaMemcpyDeviceToDevice, st));
  else
    NPFEM_CUDA_TRY(cudaMemsetAsync(g[1], 0, vb, st));
  NPFEM_CUDA_TRY(cudaMemsetAsync(gf, 0, vb, st));
  int cur = 0;  // (g[2 cur], g[2 cur + 1]) holds dL/d(x_s, v_s) of the step being reversed
  for (int sg = ncp - 1; sg >= 0; --sg) {
    const int s0 = sg * K, s1 = std::min(nsteps, s0 + K);
    NPFEM_CUDA_TRY(cudaMemcpyAsync(xw, ck + 2 * (size_t)sg * nv, vb, cudaMemcpyDeviceToDevice, st));
    NPFEM_CUDA_TRY(cudaMemcpyAsync(vw, ck + (2 * (size_t)sg + 1) * nv, vb, cudaMemcpyDeviceToDevice, st));
    for (int s = s0; s < s1; ++s) {
      NPFEM_CUDA_TRY(cudaMemcpyAsync(seg + 2 * (size_t)(s - s0) * nv, xw, vb, cudaMemcpyDeviceToDevice, st));
      NPFEM_CUDA_TRY(cudaMemcpyAsync(seg + (2 * (size_t)(s - s0) + 1) * nv, vw, vb, cudaMemcpyDeviceToDevice, st));
      if (s + 1 < s1) {
        npfem_status rc = npfem_step(b, xw, vw, f_ext, iters, &fo, nullptr, nullptr, stream);
        if (rc != NPFEM_OK) return rc;
      }
    }
    for (int s = s1 - 1; s >= s0; --s) {
      const double* xs = seg + 2 * (size_t)(s - s0) * nv;
      const double* vs = xs + nv;
      npfem_status rc = npfem_step_adjoint(b, xs, vs, f_ext, iters, opts, g[2 * cur], g[2 * cur + 1],
                                           g[2 * (1 - cur)], g[2 * (1 - cur) + 1], gfs, gwc, ssrc ? sts : nullptr,
                                           stream);
      if (rc != NPFEM_OK) return rc;
      cur = 1 - cur;
      npfem_k_add<<<grid_for((int64_t)nv), 256, 0, st>>>(gf, gfs, (int64_t)nv);
      for (const TypeLaunch& L : b->launches)
        npfem_k_type_sum<<<1, kTypeSumThreads, 0, st>>>(gwc, L.cell_list, L.ncells, gweights + 4 * L.type_index);
      if (status_out) npfem_k_or<<<grid_for(b->ncells), 256, 0, st>>>(status_out, ssrc, b->ncells);
      NPFEM_CUDA_TRY(cudaGetLastError());
    }
  }
  NPFEM_CUDA_TRY(cudaMemcpyAsync(gx0, g[2 * cur], vb, cudaMemcpyDeviceToDevice, st));
  NPFEM_CUDA_TRY(cudaMemcpyAsync(gv0, g[2 * cur + 1], vb, cudaMemcpyDeviceToDevice, st));
  return NPFEM_OK;
}

npfem_status npfem_step_adjoint_implicit(npfem_batch* b, const void* x, const void* v, const void* f_ext,
                                         const int32_t* iters, const npfem_solver_opts* opts, const double* gx_next,
                                         const double* gv_next, double* gx, double* gv, double* gf, double* gw,
                                         double cg_tol, int32_t cg_max_iters, int32_t* status_out, void* stream) {
  if (!b || !opts) return fail(NPFEM_ERR_INVALID_ARG, "step_adjoint_implicit: null batch or opts");
  if (b->prec != NPFEM_FP64) return fail(NPFEM_ERR_INVALID_ARG, "step_adjoint_implicit: needs an FP64 batch");
  if (b->ncells == 0) return NPFEM_OK;
  if (!x || !v || !f_ext || !gx_next || !gx || !gv || !gf || !gw)
    return fail(NPFEM_ERR_INVALID_ARG, "step_adjoint_implicit: null array");
  if (!(cg_tol > 0.0) || std::isinf(cg_tol) || cg_max_iters < 1)
    return fail(NPFEM_ERR_INVALID_ARG, "step_adjoint_implicit: need finite cg_tol > 0 and cg_max_iters >= 1");
  if (b->coll)
    return fail(NPFEM_ERR_INVALID_ARG,
                "step_adjoint_implicit: collisions are enabled (contacts are not differentiated)");

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t bytes = sizeof(double) * 3 * (size_t)b->n_total;
  if (!b->d_xstar) {
    void* p;
    NPFEM_CUDA_TRY(b->mem.alloc(bytes, &p));
    b->d_xstar = static_cast<double*>(p);
    NPFEM_CUDA_TRY(b->mem.alloc(bytes, &p));
    b->d_vstar = static_cast<double*>(p);
  }
  npfem_status arc = ensure_adjoint_workspace(b);
  if (arc != NPFEM_OK) return arc;
  // forward: the step on copies of x and v (x* is its final iterate)
  NPFEM_CUDA_TRY(cudaMemcpyAsync(b->d_xstar, x, bytes, cudaMemcpyDeviceToDevice, st));
  NPFEM_CUDA_TRY(cudaMemcpyAsync(b->d_vstar, v, bytes, cudaMemcpyDeviceToDevice, st));
  npfem_solver_opts o = *opts;
  o.alpha_log = nullptr;
  o.alpha_log_len = 0;
  npfem_status rc = npfem_step(b, b->d_xstar, b->d_vstar, f_ext, iters, &o, nullptr, status_out, stream);
  if (rc != NPFEM_OK) return rc;
  NPFEM_CUDA_TRY(cudaMemsetAsync(b->d_counters, 0, sizeof(int) * b->types.size() * kMaxChains * kSplitCounters, st));
  for (const TypeLaunch& L : b->launches) {
    const npfem_cell_type* t = b->types[L.type_index];
    StepParams P{};
    P.ncells_list = L.ncells;
    P.cell_list = L.cell_list;
    P.offsets = b->d_offsets;
    P.n_total = b->n_total;
    P.queue_counter = L.counter;
    P.scratch = L.scratch;
    P.slot_bytes = L.slot_bytes;
    P.z_in_smem = L.z_in_smem;
    P.solve_per_coord = L.solve_per_coord;
    P.phase_cycles = b->phase_counting ? b->d_phase : nullptr;
    ImplicitParams A{};
    A.x_n = static_cast<const double*>(x);
    A.x_star = b->d_xstar;
    A.gx_next = gx_next;
    A.gv_next = gv_next;
    A.gx = gx;
    A.gv = gv;
    A.gf = gf;
    A.gw = gw;
    A.scratch = L.adj_scratch;
    A.slot_bytes = L.adj_slot;
    A.cg_tol = cg_tol;
    A.cg_max = cg_max_iters;
    A.status_out = status_out;
    npfem_adjoint_implicit_kernel<<<L.blocks * L.warps_per_block, 32, L.smem_bytes / L.warps_per_block, st>>>(
        t->v64, P, A);  // one warp per CTA, as the unrolled adjoint
    NPFEM_CUDA_TRY(cudaGetLastError());
  }
  return NPFEM_OK;
}

npfem_status npfem_batch_set_launch(npfem_batch* b, int32_t type_index, int32_t warps_per_block,
                                    int32_t blocks_per_sm, int32_t solve_in_shared, int32_t solve_per_coord) {
  if (!b) return fail(NPFEM_ERR_INVALID_ARG, "batch_set_launch: null batch");
  NPFEM_CUDA_TRY(cudaDeviceSynchronize());
  for (TypeLaunch& L : b->launches)
    if (L.type_index == type_index)
      return configure_launch(b, L, warps_per_block, blocks_per_sm, solve_in_shared, solve_per_coord);
  return fail(NPFEM_ERR_INVALID_ARG, "batch_set_launch: no cells of that type in the batch");
}

npfem_status npfem_batch_get_launch(const npfem_batch* b, int32_t type_index, int32_t* shape) {
  if (!b || !shape) return fail(NPFEM_ERR_INVALID_ARG, "batch_get_launch: null argument");
  for (const TypeLaunch& L : b->launches)
    if (L.type_index == type_index) {
      shape[0] = L.warps_per_block;
      shape[1] = L.blocks_per_sm;
      shape[2] = L.z_in_smem;
      shape[3] = L.solve_per_coord;
      shape[4] = L.blocks;
      return NPFEM_OK;
    }
  return fail(NPFEM_ERR_INVALID_ARG, "batch_get_launch: no cells of that type in the batch");
}

npfem_status npfem_batch_set_mode(npfem_batch* b, int32_t mode) {
  if (!b || (mode != 0 && mode != 1)) return fail(NPFEM_ERR_INVALID_ARG, "batch_set_mode: mode must be 0 or 1");
  b->mode = mode;
  return NPFEM_OK;
}

npfem_status npfem_batch_set_split_launch(npfem_batch* b, int32_t type_index, const int32_t* shape) {
  if (!b || !shape) return fail(NPFEM_ERR_INVALID_ARG, "batch_set_split_launch: null argument");
  for (TypeLaunch& L : b->launches)
    if (L.type_index == type_index) {
      const HostType& H = b->types[L.type_index]->host;
      const bool cta_width = shape[2] == kCtaWarps[0] || shape[2] == kCtaWarps[1] || shape[2] == kCtaWarps[2] ||
                             shape[2] == kCtaWarps[3];
      if (shape[0] < 1 || shape[0] > 4 || shape[1] < 1 || shape[1] > 16 || shape[2] < 1 ||
          shape[2] > (shape[4] == 2 ? 8 : 4) || shape[3] < 1 || shape[3] > 16 || shape[6] < 1 || shape[6] > 4 ||
          shape[4] < 0 || shape[4] > 2)
        return fail(NPFEM_ERR_INVALID_ARG,
                    "batch_set_split_launch: warps/CTA in 1..4 (solve placement 2: 2, 4, 6 or 8), CTAs/SM in 1..16, "
                    "cells per solve warp in 1..4, placement in 0..2");
      if (shape[4] == 2 && (!cta_width || shape[5] != 0 || shape[6] < 1 || shape[6] > 2 ||
                            (shape[6] == 2 && shape[2] != kCtaWarps[0] && shape[2] != kCtaWarps[1])))
        return fail(NPFEM_ERR_INVALID_ARG,
                    "batch_set_split_launch: a CTA-cooperative solve takes 2, 4, 6 or 8 warps per CTA and one cell "
                    "(or 2 or 4 warps and two cells), interleaved coordinates");
      size_t smem = shape[4] ? split_solve_smem(H.n, shape[2], shape[5], shape[6], shape[4]) : 0;
      if (shape[4] == 2) smem += 16;  // the CTA kernel's static shared memory (rounded up)
      if (smem > (size_t)b->smem_optin)
        return fail(NPFEM_ERR_UNSUPPORTED, "batch_set_split_launch: solve vectors exceed shared memory");
      L.it_wpb = shape[0];
      L.it_bps = shape[1];
      L.sv_wpb = shape[2];
      L.sv_bps = shape[3];
      L.sv_smem = shape[4];
      L.sv_percoord = shape[5] ? 1 : 0;
      L.sv_cells = shape[6];
      return NPFEM_OK;
    }
  return fail(NPFEM_ERR_INVALID_ARG, "batch_set_split_launch: no cells of that type in the batch");
}

npfem_status npfem_batch_get_split_launch(const npfem_batch* b, int32_t type_index, int32_t* shape) {
  if (!b || !shape) return fail(NPFEM_ERR_INVALID_ARG, "batch_get_split_launch: null argument");
  for (const TypeLaunch& L : b->launches)
    if (L.type_index == type_index) {
      shape[0] = L.it_wpb;
      shape[1] = L.it_bps;
      shape[2] = L.sv_wpb;
      shape[3] = L.sv_bps;
      shape[4] = L.sv_smem;
      shape[5] = L.sv_percoord;
      shape[6] = L.sv_cells;
      shape[7] = b->mode;
      return NPFEM_OK;
    }
  return fail(NPFEM_ERR_INVALID_ARG, "batch_get_split_launch: no cells of that type in the batch");
}

npfem_status npfem_batch_set_phase_counting(npfem_batch* b, int32_t enable) {
  if (!b) return fail(NPFEM_ERR_INVALID_ARG, "batch_set_phase_counting: null batch");
  b->phase_counting = enable != 0;
  return NPFEM_OK;
}

npfem_status npfem_batch_phase_cycles(npfem_batch* b, uint64_t* cycles, int32_t reset) {
  if (!b || !cycles) return fail(NPFEM_ERR_INVALID_ARG, "batch_phase_cycles: null argument");
  NPFEM_CUDA_TRY(cudaDeviceSynchronize());
  unsigned long long h[kPhases];
  NPFEM_CUDA_TRY(cudaMemcpy(h, b->d_phase, sizeof(h), cudaMemcpyDeviceToHost));
  for (int k = 0; k < kPhases; ++k) cycles[k] = h[k];
  if (reset) NPFEM_CUDA_TRY(cudaMemset(b->d_phase, 0, sizeof(h)));
  return NPFEM_OK;
}

npfem_status npfem_batch_set_kernel_timing(npfem_batch* b, int32_t enable) {
  if (!b) return fail(NPFEM_ERR_INVALID_ARG, "batch_set_kernel_timing: null batch");
  const size_t chains = b->launches.size() * kMaxChains;
  if (enable && b->kev.size() < chains * kTimingSlots * 2) {
    const size_t old = b->kev.size();
    b->kev.resize(chains * kTimingSlots * 2, nullptr);
    for (size_t i = old; i < b->kev.size(); ++i) NPFEM_CUDA_TRY(cudaEventCreate(&b->kev[i]));
    b->k_last_slots.assign(chains, 0);
  }
  if (enable && !b->k_ref) NPFEM_CUDA_TRY(cudaEventCreate(&b->k_ref));
  if (enable)
    for (cudaEvent_t& e : b->det_ev)
      if (!e) NPFEM_CUDA_TRY(cudaEventCreate(&e));
  b->ktiming = enable != 0 && !b->launches.empty();
  return NPFEM_OK;
}

npfem_status npfem_batch_contact_time(npfem_batch* b, double* ms) {
  if (!b || !ms) return fail(NPFEM_ERR_INVALID_ARG, "batch_contact_time: null argument");
  *ms = 0.0;
  if (!b->det_timed)
    return fail(NPFEM_ERR_INVALID_ARG, "batch_contact_time: the last step was not timed with collisions on");
  NPFEM_CUDA_TRY(cudaEventSynchronize(b->det_ev[1]));
  float t = 0.f;
  NPFEM_CUDA_TRY(cudaEventElapsedTime(&t, b->det_ev[0], b->det_ev[1]));
  *ms = t;
  return NPFEM_OK;
}

npfem_status npfem_batch_kernel_times(npfem_batch* b, int32_t type_index, double* ms, int32_t* launches) {
  if (!b || !ms || !launches) return fail(NPFEM_ERR_INVALID_ARG, "batch_kernel_times: null argument");
  for (int k = 0; k < 3; ++k) ms[k] = 0.0, launches[k] = 0;
  if (b->kev.empty()) return fail(NPFEM_ERR_INVALID_ARG, "batch_kernel_times: kernel timing was never enabled");
  bool found = false;
  for (const TypeLaunch& L : b->launches) found = found || L.type_index == type_index;
  if (!found) return fail(NPFEM_ERR_INVALID_ARG, "batch_kernel_times: no cells of that type in the batch");
  for (size_t c = 0; c < b->k_last_chains.size() && c < b->k_last_slots.size(); ++c) {
    if (b->k_last_chains[c] != type_index) continue;
    for (int slot = 0; slot < b->k_last_slots[c]; ++slot) {
      cudaEvent_t* ke = &b->kev[(c * kTimingSlots + slot) * 2];
      NPFEM_CUDA_TRY(cudaEventSynchronize(ke[1]));
      float t = 0.f;
      NPFEM_CUDA_TRY(cudaEventElapsedTime(&t, ke[0], ke[1]));
      const int kind = slot == 0 ? 0 : 2 - (slot & 1);
      ms[kind] += t;
      launches[kind] += 1;
    }
  }
  return NPFEM_OK;
}

npfem_status npfem_batch_kernel_spans(npfem_batch* b, int32_t type_index, double* span_ms) {
  if (!b || !span_ms) return fail(NPFEM_ERR_INVALID_ARG, "batch_kernel_spans: null argument");
  for (int k = 0; k < 3; ++k) span_ms[k] = 0.0;
  if (b->kev.empty() || !b->k_ref)
    return fail(NPFEM_ERR_INVALID_ARG, "batch_kernel_spans: kernel timing was never enabled");
  // launch intervals relative to the step's reference event, per kernel kind
  std::vector<std::pair<double, double>> iv[3];
  for (size_t c = 0; c < b->k_last_chains.size() && c < b->k_last_slots.size(); ++c) {
    if (type_index >= 0 && b->k_last_chains[c] != type_index) continue;
    for (int slot = 0; slot < b->k_last_slots[c]; ++slot) {
      cudaEvent_t* ke = &b->kev[(c * kTimingSlots + slot) * 2];
      NPFEM_CUDA_TRY(cudaEventSynchronize(ke[1]));
      float t0 = 0.f, t1 = 0.f;
      NPFEM_CUDA_TRY(cudaEventElapsedTime(&t0, b->k_ref, ke[0]));
      NPFEM_CUDA_TRY(cudaEventElapsedTime(&t1, b->k_ref, ke[1]));
      iv[slot == 0 ? 0 : 2 - (slot & 1)].push_back({t0, t1});
    }
  }
  for (int k = 0; k < 3; ++k) {  // length of the union of the intervals
    std::sort(iv[k].begin(), iv[k].end());
    double end = -1e300, total = 0.0;
    for (const auto& q : iv[k]) {
      if (q.first > end) {
        total += q.second - q.first;
        end = q.second;
      } else if (q.second > end) {
        total += q.second - end;
        end = q.second;
      }
    }
    span_ms[k] = total;
  }
  return NPFEM_OK;
}

npfem_status npfem_batch_set_groups(npfem_batch* b, int32_t type_index, int32_t groups) {
  if (!b || groups < 1 || groups > kMaxGroups)
    return fail(NPFEM_ERR_INVALID_ARG, "batch_set_groups: groups in 1..4");
  for (TypeLaunch& L : b->launches)
    if (L.type_index == type_index) {
      L.groups = groups;
      return NPFEM_OK;
    }
  return fail(NPFEM_ERR_INVALID_ARG, "batch_set_groups: no cells of that type in the batch");
}

npfem_status npfem_batch_get_groups(const npfem_batch* b, int32_t type_index, int32_t* groups) {
  if (!b || !groups) return fail(NPFEM_ERR_INVALID_ARG, "batch_get_groups: null argument");
  for (const TypeLaunch& L : b->launches)
    if (L.type_index == type_index) {
      *groups = L.groups;
      return NPFEM_OK;
    }
  return fail(NPFEM_ERR_INVALID_ARG, "batch_get_groups: no cells of that type in the batch");
}

npfem_status npfem_batch_set_solve_streams(npfem_batch* b, int32_t enable) {
  if (!b) return fail(NPFEM_ERR_INVALID_ARG, "batch_set_solve_streams: null batch");
  NPFEM_CUDA_TRY(cudaDeviceSynchronize());
  b->solve_streams_on = enable != 0;
  return NPFEM_OK;
}

npfem_status npfem_batch_set_iter_width(npfem_batch* b, int32_t type_index, int32_t warps) {
  if (!b || warps < 0 || warps > kIterCtaMaxWarps || (warps & (warps - 1)) != 0)
    return fail(NPFEM_ERR_INVALID_ARG, "batch_set_iter_width: warps in 0, 1, 2, 4, 8, 16");
  for (TypeLaunch& L : b->launches)
    if (L.type_index == type_index) {
      const int keep_w = L.itc_w, keep_b = L.itc_bps;
      if (!set_iter_cta(b, L, warps)) {
        L.itc_w = keep_w;
        L.itc_bps = keep_b;
        return fail(NPFEM_ERR_UNSUPPORTED,
                    "batch_set_iter_width: the type's shared-memory arrays exceed a CTA, or its elements are not "
                    "coloured");
      }
      return NPFEM_OK;
    }
  return fail(NPFEM_ERR_INVALID_ARG, "batch_set_iter_width: no cells of that type in the batch");
}

npfem_status npfem_batch_get_iter_width(const npfem_batch* b, int32_t type_index, int32_t* warps,
                                        int32_t* ctas_per_sm) {
  if (!b || !warps) return fail(NPFEM_ERR_INVALID_ARG, "batch_get_iter_width: null argument");
  for (const TypeLaunch& L : b->launches)
    if (L.type_index == type_index) {
      *warps = L.itc_w;
      if (ctas_per_sm) *ctas_per_sm = L.itc_bps;
      return NPFEM_OK;
    }
  return fail(NPFEM_ERR_INVALID_ARG, "batch_get_iter_width: no cells of that type in the batch");
}

npfem_status npfem_step_host(npfem_batch* b, void* x, void* v, const void* f_ext, const int32_t* iters,
                             const npfem_solver_opts* opts, double* residual_out, int32_t* status_out,
                             void* stream) {
  if (!b || !opts || !x || !v || !f_ext) return fail(NPFEM_ERR_INVALID_ARG, "step_host: null argument");
  if (b->ncells == 0) return NPFEM_OK;
  if (!(opts->tol >= 0.0) || std::isinf(opts->tol))
    return fail(NPFEM_ERR_INVALID_ARG, "step_host: tol must be finite and >= 0");
  const size_t ssize = b->prec == NPFEM_FP64 ? sizeof(double) : sizeof(float);
  const size_t bytes = ssize * 3 * (size_t)b->n_total;
  if (!b->d_x) {
    void* p;
    NPFEM_CUDA_TRY(b->mem.alloc(bytes, &p));
    b->d_x = p;
    NPFEM_CUDA_TRY(b->mem.alloc(bytes, &p));
    b->d_v = p;
    NPFEM_CUDA_TRY(b->mem.alloc(bytes, &p));
    b->d_f = p;
    NPFEM_CUDA_TRY(b->mem.alloc(sizeof(int32_t) * b->ncells, &p));
    b->d_iters = static_cast<int32_t*>(p);
    NPFEM_CUDA_TRY(b->mem.alloc(sizeof(double) * b->ncells, &p));
    b->d_res = static_cast<double*>(p);
    NPFEM_CUDA_TRY(b->mem.alloc(sizeof(int32_t) * b->ncells, &p));
    b->d_status = static_cast<int32_t*>(p);
    NPFEM_CUDA_TRY(b->mem.alloc(sizeof(int32_t) * b->ncells, &p));
    b->d_done = static_cast<int32_t*>(p);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  npfem_solver_opts o = *opts;
  o.alpha_log = nullptr;
  o.alpha_log_len = 0;
  o.iters_done = opts->iters_done ? b->d_done : nullptr;
  int max_iters = 0;
  bool split = b->mode == 1 && (iters == nullptr || opts->max_iters > 0);
  if (split) {
    max_iters = iters ? opts->max_iters : opts->iters;
    split = max_iters <= kSplitMaxIters && max_iters >= 0;
  }
  // chunks: up to 12 chains in all (8 chunks for one cell type, 4 for three)
  const int per_type = std::max(2, 12 / std::max(1, (int)b->launches.size()));
  // contact detection needs every cell's input on the device: one chunk with collisions
  const int K = split && !b->coll ? std::min(std::min(kMaxChains, per_type), b->ncells) : 1;
  if (K < 2) {  // one chunk: copies in, step, copies out
    NPFEM_CUDA_TRY(cudaMemcpyAsync(b->d_x, x, bytes, cudaMemcpyHostToDevice, st));
    NPFEM_CUDA_TRY(cudaMemcpyAsync(b->d_v, v, bytes, cudaMemcpyHostToDevice, st));
    NPFEM_CUDA_TRY(cudaMemcpyAsync(b->d_f, f_ext, bytes, cudaMemcpyHostToDevice, st));
    if (iters)
      NPFEM_CUDA_TRY(cudaMemcpyAsync(b->d_iters, iters, sizeof(int32_t) * b->ncells, cudaMemcpyHostToDevice, st));
    npfem_status rc = npfem_step(b, b->d_x, b->d_v, b->d_f, iters ? b->d_iters : nullptr, &o, b->d_res,
                                 b->d_status, stream);
    if (rc != NPFEM_OK) return rc;
    NPFEM_CUDA_TRY(cudaMemcpyAsync(x, b->d_x, bytes, cudaMemcpyDeviceToHost, st));
    NPFEM_CUDA_TRY(cudaMemcpyAsync(v, b->d_v, bytes, cudaMemcpyDeviceToHost, st));
  } else {
    // K chunks of consecutive cells (about equal vertex counts): chunk g's inputs are
    // copied on the copy-in stream, its chains start when they have arrived, and its
    // outputs are copied back on the copy-out stream as soon as its chains are done, so
    // copies overlap the other chunks' kernels.
    const size_t nl = b->launches.size();
    const size_t nev = 2 + kMaxChains + kMaxChains * nl;
    if (!b->h2d_stream) NPFEM_CUDA_TRY(cudaStreamCreateWithFlags(&b->h2d_stream, cudaStreamNonBlocking));
    if (!b->d2h_stream) NPFEM_CUDA_TRY(cudaStreamCreateWithFlags(&b->d2h_stream, cudaStreamNonBlocking));
    while (b->pipe_events.size() < nev) {
      cudaEvent_t e;
      NPFEM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      b->pipe_events.push_back(e);
    }
    cudaEvent_t* ev_start = &b->pipe_events[0];
    cudaEvent_t* ev_in = &b->pipe_events[1];
    cudaEvent_t* ev_done = &b->pipe_events[1 + kMaxChains];
    cudaEvent_t* ev_out = &b->pipe_events[1 + kMaxChains + kMaxChains * nl];
    int bounds[kMaxChains + 1];
    bounds[0] = 0;
    for (int g = 1; g < K; ++g) {
      const int64_t target = b->n_total * g / K;
      int c = (int)(std::lower_bound(b->offsets.begin(), b->offsets.end() - 1, target) - b->offsets.begin());
      bounds[g] = std::max(bounds[g - 1], std::min(c, b->ncells));
    }
    bounds[K] = b->ncells;
    const int64_t Nt = b->n_total;
    auto part = [&](const void* base, int64_t o0) { return static_cast<const char*>(base) + ssize * o0; };
    auto partw = [&](void* base, int64_t o0) { return static_cast<char*>(base) + ssize * o0; };
    NPFEM_CUDA_TRY(cudaEventRecord(*ev_start, st));
    NPFEM_CUDA_TRY(cudaStreamWaitEvent(b->h2d_stream, *ev_start, 0));
    NPFEM_CUDA_TRY(cudaStreamWaitEvent(b->d2h_stream, *ev_start, 0));
    if (iters)
      NPFEM_CUDA_TRY(
          cudaMemcpyAsync(b->d_iters, iters, sizeof(int32_t) * b->ncells, cudaMemcpyHostToDevice, b->h2d_stream));
    for (int g = 0; g < K; ++g) {
      const int64_t o0 = b->offsets[bounds[g]], o1 = b->offsets[bounds[g + 1]];
      const size_t nb = ssize * (size_t)(o1 - o0);
      if (nb)
        for (int d = 0; d < 3; ++d) {
          NPFEM_CUDA_TRY(cudaMemcpyAsync(partw(b->d_x, d * Nt + o0), part(x, d * Nt + o0), nb,
                                         cudaMemcpyHostToDevice, b->h2d_stream));
          NPFEM_CUDA_TRY(cudaMemcpyAsync(partw(b->d_v, d * Nt + o0), part(v, d * Nt + o0), nb,
                                         cudaMemcpyHostToDevice, b->h2d_stream));
          NPFEM_CUDA_TRY(cudaMemcpyAsync(partw(b->d_f, d * Nt + o0), part(f_ext, d * Nt + o0), nb,
                                         cudaMemcpyHostToDevice, b->h2d_stream));
        }
      NPFEM_CUDA_TRY(cudaEventRecord(ev_in[g], b->h2d_stream));
    }
    PipelinePlan plan{K, bounds, ev_in, ev_done};
    npfem_status rc = step_split(b, b->d_x, b->d_v, b->d_f, iters ? b->d_iters : nullptr, &o, max_iters, b->d_res,
                                 b->d_status, st, &plan);
    if (rc != NPFEM_OK) return rc;
    for (int g = 0; g < K; ++g) {
      for (size_t li = 0; li < nl; ++li)
        NPFEM_CUDA_TRY(cudaStreamWaitEvent(b->d2h_stream, ev_done[g * nl + li], 0));
      const int64_t o0 = b->offsets[bounds[g]], o1 = b->offsets[bounds[g + 1]];
      const size_t nb = ssize * (size_t)(o1 - o0);
      if (nb)
        for (int d = 0; d < 3; ++d) {
          NPFEM_CUDA_TRY(cudaMemcpyAsync(partw(x, d * Nt + o0), part(b->d_x, d * Nt + o0), nb,
                                         cudaMemcpyDeviceToHost, b->d2h_stream));
          NPFEM_CUDA_TRY(cudaMemcpyAsync(partw(v, d * Nt + o0), part(b->d_v, d * Nt + o0), nb,
                                         cudaMemcpyDeviceToHost, b->d2h_stream));
        }
    }
    NPFEM_CUDA_TRY(cudaEventRecord(*ev_out, b->d2h_stream));
    NPFEM_CUDA_TRY(cudaStreamWaitEvent(st, *ev_out, 0));
  }
  if (residual_out)
    NPFEM_CUDA_TRY(cudaMemcpyAsync(residual_out, b->d_res, sizeof(double) * b->ncells, cudaMemcpyDeviceToHost, st));
  if (status_out)
    NPFEM_CUDA_TRY(
        cudaMemcpyAsync(status_out, b->d_status, sizeof(int32_t) * b->ncells, cudaMemcpyDeviceToHost, st));
  if (opts->iters_done)
    NPFEM_CUDA_TRY(cudaMemcpyAsync(opts->iters_done, b->d_done, sizeof(int32_t) * b->ncells,
                                   cudaMemcpyDeviceToHost, st));
  NPFEM_CUDA_TRY(cudaStreamSynchronize(st));
  return NPFEM_OK;
}

npfem_status npfem_batch_set_collisions(npfem_batch* b, const npfem_collision_params* p) {
  if (!b) return fail(NPFEM_ERR_INVALID_ARG, "batch_set_collisions: null batch");
  if (!p) {
    b->coll = false;
    return NPFEM_OK;
  }
  if (!(p->radius > 0.0) || std::isinf(p->radius) || !(p->delta >= 0.0) || std::isinf(p->delta) ||
      !(p->weight >= 0.0) || std::isinf(p->weight))
    return fail(NPFEM_ERR_INVALID_ARG, "batch_set_collisions: need finite radius > 0, delta >= 0, weight >= 0");
  if (p->walls)
    for (int d = 0; d < 3; ++d)
      if (!(p->box_lo[d] < p->box_hi[d]) || std::isinf(p->box_lo[d]) || std::isinf(p->box_hi[d]))
        return fail(NPFEM_ERR_INVALID_ARG, "batch_set_collisions: walls need a finite box with box_lo < box_hi");
  if (b->n_total >= ((int64_t)1 << 30))
    return fail(NPFEM_ERR_UNSUPPORTED, "batch_set_collisions: more than 2^30 vertices");
  size_t nsmem = 0;  // the normals kernel keeps a cell's triangle normals in shared memory
  for (const npfem_cell_type* t : b->types) nsmem = std::max(nsmem, sizeof(double) * 3 * (size_t)t->host.T);
  if (nsmem > (size_t)b->smem_optin)
    return fail(NPFEM_ERR_UNSUPPORTED, "batch_set_collisions: a cell type has too many triangles for the "
                                       "normals kernel's shared memory (" + std::to_string(nsmem) + " bytes)");
  // the attribute is per kernel, shared by every batch: the device maximum serves them all
  NPFEM_CUDA_TRY(cudaFuncSetAttribute(npfem_k_normals<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      b->smem_optin));
  NPFEM_CUDA_TRY(cudaFuncSetAttribute(npfem_k_normals<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      b->smem_optin));
  if (!b->coll_alloc && b->n_total > 0) {
    const int64_t N = b->n_total;
    int64_t T = kScanBlock;
    while (T < N) T <<= 1;
    ContactParams& C = b->cp;
    void* q = nullptr;
    auto take = [&](size_t bytes, void** out) -> cudaError_t { return b->mem.alloc(bytes, out); };
    NPFEM_CUDA_TRY(take(sizeof(int32_t) * N, &q));
    C.vcell = static_cast<const int32_t*>(q);
    int32_t* vcell = static_cast<int32_t*>(q);
    NPFEM_CUDA_TRY(take(sizeof(int32_t) * N, &q));
    C.key = static_cast<int32_t*>(q);
    NPFEM_CUDA_TRY(take(sizeof(int32_t) * T, &q));
    C.count = static_cast<int32_t*>(q);
    NPFEM_CUDA_TRY(take(sizeof(int32_t) * (T + 1), &q));
    C.start = static_cast<int32_t*>(q);
    NPFEM_CUDA_TRY(take(sizeof(int32_t) * T, &q));
    C.cursor = static_cast<int32_t*>(q);
    NPFEM_CUDA_TRY(take(sizeof(int32_t) * (T / kScanBlock), &q));
    C.bsum = static_cast<int32_t*>(q);
    NPFEM_CUDA_TRY(take(sizeof(int32_t) * N, &q));
    C.sorted = static_cast<int32_t*>(q);
    NPFEM_CUDA_TRY(take(sizeof(float4) * N, &q));
    C.sortpos = static_cast<float4*>(q);
    NPFEM_CUDA_TRY(take(256, &q));
    C.maxabs = static_cast<int32_t*>(q);
    NPFEM_CUDA_TRY(take(sizeof(double) * 6, &q));
    C.box = static_cast<double*>(q);
    NPFEM_CUDA_TRY(take(sizeof(double) * 3 * N, &q));
    C.nrm = static_cast<double*>(q);
    NPFEM_CUDA_TRY(take(sizeof(int32_t) * N, &q));
    C.ccount = static_cast<int32_t*>(q);
    NPFEM_CUDA_TRY(take(sizeof(int32_t) * kContactSlots * N, &q));
    C.cvertex = static_cast<int32_t*>(q);
    NPFEM_CUDA_TRY(take(sizeof(double) * 4 * kContactSlots * N, &q));
    C.cplane = static_cast<double*>(q);
    C.offsets = b->d_offsets;
    std::vector<int32_t> hv((size_t)N);
    for (int c = 0; c < b->ncells; ++c)
      for (int64_t i = b->offsets[c]; i < b->offsets[c + 1]; ++i) hv[(size_t)i] = c;
    NPFEM_CUDA_TRY(cudaMemcpy(vcell, hv.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice));
    b->coll_T = T;
    b->coll_alloc = true;
  }
  b->coll_p = *p;
  b->coll = true;
  if (b->coll_alloc && p->walls) {
    const double box[6] = {p->box_lo[0], p->box_lo[1], p->box_lo[2], p->box_hi[0], p->box_hi[1], p->box_hi[2]};
    NPFEM_CUDA_TRY(cudaMemcpy(b->cp.box, box, sizeof(box), cudaMemcpyHostToDevice));
  }
  return NPFEM_OK;
}

npfem_status npfem_batch_contacts(npfem_batch* b, int32_t* count, int32_t* vertex, double* plane, void* stream) {
  if (!b) return fail(NPFEM_ERR_INVALID_ARG, "batch_contacts: null batch");
  if (b->n_total == 0) return NPFEM_OK;
  if (!b->coll_alloc) return fail(NPFEM_ERR_INVALID_ARG, "batch_contacts: collisions were never enabled");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t N = b->n_total;
  if (count)
    NPFEM_CUDA_TRY(cudaMemcpyAsync(count, b->cp.ccount, sizeof(int32_t) * N, cudaMemcpyDeviceToDevice, st));
  if (vertex)
    NPFEM_CUDA_TRY(cudaMemcpyAsync(vertex, b->cp.cvertex, sizeof(int32_t) * kContactSlots * N,
                                   cudaMemcpyDeviceToDevice, st));
  if (plane)
    NPFEM_CUDA_TRY(cudaMemcpyAsync(plane, b->cp.cplane, sizeof(double) * 4 * kContactSlots * N,
                                   cudaMemcpyDeviceToDevice, st));
  return NPFEM_OK;
}

}  // extern "C"
