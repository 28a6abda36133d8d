// The batched step as a sequence of kernels (split mode): the same per-cell arithmetic as
// process_cell, cut at the global solves so that the FP64 triangular sweeps run in a kernel
// of their own.
//
//   k_begin   K1 prediction, first objective evaluation, first half of the two-loop (Q = g)
//   k_solve   Q <- A^-1 Q, FP64 LDL^T sweeps with the solve vector in shared memory
//   k_iter    second half of the two-loop, line search, history update, then either the
//             first half of the next iteration's two-loop or the K7 write-back
//
// One step launches k_begin once and (k_solve, k_iter) max_iters times per cell type.
// Between kernels each cell's state lives in its own workspace slot (a CellState header
// followed by the CellWs vectors and a workspace copy of the solve vector, used only by
// the rare non-descent reset inside k_iter).  k_iter and the CTA-cooperative solve walk
// the group's cells in batch order and skip those whose step has ended (budget used, or
// tolerance met in the converged-residual mode): measured faster than taking them from
// the compacted list of the cells still iterating, whose order is that in which the
// previous kernel finished them.  The one-warp solve, which packs several cells per
// warp, takes its cells from that list (written by k_begin for iteration 0 and by
// k_iter(i - 1) for iteration i).
#pragma once
#include "step_kernel.cuh"

namespace npfem {

constexpr int kSplitMaxIters = 32;
// Resident 128-thread CTAs per SM that k_begin and k_iter are compiled for (a budget of
// 65536 / (128 x min_blocks) registers per thread).  The FP32 form is bound by the
// latency of its gathers, not by arithmetic: 64 registers let 32 warps per SM hold one
// cell each (4096 cells in one wave instead of two at 16 warps).  The FP64 objective
// is bound by the FP64 pipe from 12 warps per SM on: 128 registers, 16 warps.
template <typename S>
struct IterOccupancy {
  static constexpr int min_blocks = 4;
};
template <>
struct IterOccupancy<float> {
  static constexpr int min_blocks = 8;
};

// Device counters per cell type and step: [0] k_begin queue, [1 + 2i] / [2 + 2i] queues of
// k_solve / k_iter of iteration i, [kActiveCountOff + i] length of the list of cells
// that still iterate at iteration i (appended by k_begin for i = 0, by k_iter(i - 1)).
constexpr int kActiveCountOff = 2 + 2 * kSplitMaxIters;
constexpr int kSplitCounters = kActiveCountOff + kSplitMaxIters + 1;
// A type's cells run as up to kMaxChains chains of kernels, each with its own counter
// block: up to kMaxGroups concurrent groups of a device-buffer step, up to kMaxChains
// chunks of a pipelined host-buffer step.
constexpr int kMaxGroups = 4;
constexpr int kMaxChains = 8;
constexpr size_t kStateBytes = 256;

template <typename S>
struct CellState {
  double fx, g0n;
  int k, iters, hcount, hhead, status, degen, cur;  // cur: 1 when UT/GT hold the current iterate
  S rho[kHistory], aco[kHistory];
  S cvol[3];
};
static_assert(sizeof(CellState<double>) <= kStateBytes, "cell state header too large");

struct SplitCtx {
  char* base;
  int cell;
};

template <typename S>
__device__ __forceinline__ CellWs<S> split_ws(char* base, const DevTypeView<S>& ty) {
  return carve<S>(base + kStateBytes, ty.n, ty.T, ty.E, nullptr);
}

// Fused streaming passes of the two-loop recursion.  Each lane (thread) takes the
// elements lane, lane + stride, ... in increasing order (the order of a separate pass;
// stride 32 for a warp, the CTA size for a CTA), four at a time with every load of the
// four issued before the first store, so the loads of a pass stay in flight together
// although the pass writes one of the vectors it reads.
template <typename S>
__device__ __forceinline__ S update_dot(S* q, S c, const S* u, const S* t, int len, int lane, int stride = 32) {
  // q += c u; returns this lane's partial sum of t . q over the updated values
  S acc = 0;
  int e = lane;
  for (; e + 3 * stride < len; e += 4 * stride) {
    S qv[4], uv[4], tv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      qv[j] = q[e + stride * j];
      uv[j] = u[e + stride * j];
      tv[j] = t[e + stride * j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const S qn = qv[j] + c * uv[j];
      q[e + stride * j] = qn;
      acc += tv[j] * qn;
    }
  }
  for (; e < len; e += stride) {
    const S qn = q[e] + c * u[e];
    q[e] = qn;
    acc += t[e] * qn;
  }
  return acc;
}

template <typename S>
__device__ __forceinline__ S copy_dot(S* q, const S* g, const S* t, int len, int lane, int stride = 32) {
  // q = g; returns this lane's partial sum of t . g
  S acc = 0;
  int e = lane;
  for (; e + 3 * stride < len; e += 4 * stride) {
    S gv[4], tv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      gv[j] = g[e + stride * j];
      tv[j] = t[e + stride * j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      q[e + stride * j] = gv[j];
      acc += tv[j] * gv[j];
    }
  }
  for (; e < len; e += stride) {
    const S gq = g[e];
    q[e] = gq;
    acc += t[e] * gq;
  }
  return acc;
}

template <typename S>
__device__ __forceinline__ void update_negate(const S* q, S c, const S* u, const S* g, S* d, Acc<S>& agd, int len,
                                              int lane) {
  // d = -(q + c u); agd accumulates g . d
  int e = lane;
  for (; e + 96 < len; e += 128) {
    S qv[4], uv[4], gv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      qv[j] = q[e + 32 * j];
      uv[j] = u[e + 32 * j];
      gv[j] = g[e + 32 * j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const S dv = -(qv[j] + c * uv[j]);
      d[e + 32 * j] = dv;
      agd.add_prod(gv[j], dv);
    }
  }
  for (; e < len; e += 32) {
    const S dv = -(q[e] + c * u[e]);
    d[e] = dv;
    agd.add_prod(g[e], dv);
  }
}

// First half of the two-loop recursion: Q = g, newest -> oldest pairs.  Each pass applies
// one pair's update and accumulates the next pair's s . Q from the updated values it holds
// in registers, so Q is read once per pair (the products and each lane's summation order
// are those of separate dot and update passes).
template <typename S>
__device__ __forceinline__ void two_loop_first(const CellWs<S>& w, CellState<S>* st, const S* G, int len,
                                               int lane) {
  const int hc = st->hcount, hh = st->hhead;
  if (hc == 0) {
    for (int e = lane; e < len; e += 32) w.Q[e] = G[e];
    __syncwarp();
    return;
  }
  int i = (hh - 1 + kHistory) % kHistory;
  S acc = copy_dot<S>(w.Q, G, w.hs + (size_t)i * len, len, lane);
  for (int q = 0; q < hc; ++q) {
    const S a = st->rho[i] * warp_sum<S>(acc);
    if (lane == 0) st->aco[i] = a;
    const S* yi = w.hy + (size_t)i * len;
    if (q + 1 < hc) {
      const int inext = (hh - 1 - (q + 1) + kHistory) % kHistory;
      acc = update_dot<S>(w.Q, -a, yi, w.hs + (size_t)inext * len, len, lane);
      i = inext;
    } else {
      for (int e = lane; e < len; e += 32) w.Q[e] -= a * yi[e];
    }
  }
  __syncwarp();
}

// K7: residual, x_{n+1} = anchor + X + U, v_{n+1} = U / dt, status.
template <typename S>
__device__ void split_finalize(const DevTypeView<S>& ty, const StepParams& P, const CellWs<S>& w, CellState<S>* st,
                               const S* U, const S* G, int cell, int done, S* x, S* v, int lane) {
  const int n = ty.n, len = 3 * n;
  const int64_t off = P.offsets[cell], Nt = P.n_total;
  NPFEM_PHASE_BEGIN(t_write)
  const S ax = x[off], ay = x[Nt + off], az = x[2 * Nt + off];
  const double gn = sqrt(vdot64<S>(G, G, len, lane));
  const S idt = (S)(1.0 / ty.dt);
  bool bad = false;
  __syncwarp();
  for (int k = lane; k < n; k += 32) {
    double nx = (double)ax + ((double)w.X[3 * k] + (double)U[3 * k]);
    double ny = (double)ay + ((double)w.X[3 * k + 1] + (double)U[3 * k + 1]);
    double nz = (double)az + ((double)w.X[3 * k + 2] + (double)U[3 * k + 2]);
    S vx = U[3 * k] * idt, vy = U[3 * k + 1] * idt, vz = U[3 * k + 2] * idt;
    bad = bad || !isfinite(nx) || !isfinite(ny) || !isfinite(nz) || !isfinite((double)vx) ||
          !isfinite((double)vy) || !isfinite((double)vz);
    if (k != 0) {
      x[off + k] = (S)nx;
      x[Nt + off + k] = (S)ny;
      x[2 * Nt + off + k] = (S)nz;
    }
    v[off + k] = vx;
    v[Nt + off + k] = vy;
    v[2 * Nt + off + k] = vz;
  }
  // vertex 0 is the anchor: every lane read it above, so it is written last
  __syncwarp();
  if (lane == 0) {
    double nx = (double)ax + ((double)w.X[0] + (double)U[0]);
    double ny = (double)ay + ((double)w.X[1] + (double)U[1]);
    double nz = (double)az + ((double)w.X[2] + (double)U[2]);
    x[off] = (S)nx;
    x[Nt + off] = (S)ny;
    x[2 * Nt + off] = (S)nz;
  }
  bad = __any_sync(kFull, bad);
  NPFEM_PHASE_END(t_write, kPhWrite, P, lane)
  if (lane == 0) {
    int status = st->status;
    if (st->degen) status |= 2;
    if (bad) status |= 4;
    if (P.status_out) P.status_out[cell] = status;
    if (P.residual_out) P.residual_out[cell] = st->g0n > 0.0 ? gn / st->g0n : 0.0;
    if (P.iters_done) P.iters_done[cell] = done;
    st->k = st->iters;
  }
  __syncwarp();
}

template <typename S, bool kLim>
__global__ void __launch_bounds__(128, IterOccupancy<S>::min_blocks) npfem_k_begin(DevTypeView<S> ty, StepParams P, int max_iters, S* x,
                                                     S* v, const S* f) {
  const int lane = threadIdx.x & 31;
  const int n = ty.n, len = 3 * n;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(P.queue_counter, 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= P.ncells_list) break;
    const int cell = P.cell_list[item];
    char* base = P.scratch + (size_t)item * P.slot_bytes;
    CellState<S>* st = reinterpret_cast<CellState<S>*>(base);
    CellWs<S> w = split_ws<S>(base, ty);
    const int64_t off = P.offsets[cell], Nt = P.n_total;
    int iters = P.iters ? P.iters[cell] : P.iters_default;
    int status = 0;
    if (iters > max_iters) {
      iters = max_iters;
      status |= 8;
    }
    if (iters < 0) iters = 0;
    const double dt = ty.dt;
    const S sdt = (S)dt, sdt2 = (S)(dt * dt);
    NPFEM_PHASE_BEGIN(t_predict)
    const S ax = x[off], ay = x[Nt + off], az = x[2 * Nt + off];
    Acc<S> cx, cy, cz;
    for (int k = lane; k < n; k += 32) {
      S px = x[off + k] - ax, py = x[Nt + off + k] - ay, pz = x[2 * Nt + off + k] - az;
      w.X[3 * k] = px;
      w.X[3 * k + 1] = py;
      w.X[3 * k + 2] = pz;
      cx.add(px);
      cy.add(py);
      cz.add(pz);
      const S im = __ldg(&ty.inv_mass[k]);
      S wx = sdt * v[off + k] + sdt2 * f[off + k] * im;
      S wy = sdt * v[Nt + off + k] + sdt2 * f[Nt + off + k] * im;
      S wz = sdt * v[2 * Nt + off + k] + sdt2 * f[2 * Nt + off + k] * im;
      w.W[3 * k] = wx;
      w.W[3 * k + 1] = wy;
      w.W[3 * k + 2] = wz;
      w.U[3 * k] = wx;
      w.U[3 * k + 1] = wy;
      w.U[3 * k + 2] = wz;
    }
    V3<S> cvol{(S)(cx.total() / n), (S)(cy.total() / n), (S)(cz.total() / n)};
    __syncwarp();
    NPFEM_PHASE_END(t_predict, kPhPredict, P, lane)
    NPFEM_PHASE_BEGIN(t_obj0)
    EvalOut ev = eval_objective<S, kLim ? 1 : 0>(ty, P, w, w.U, w.G, cvol, cell, lane);
    NPFEM_PHASE_END(t_obj0, kPhObjective, P, lane)
    const double g0n = sqrt(vdot64<S>(w.G, w.G, len, lane));
    if (lane == 0) {
      st->fx = ev.energy;
      st->g0n = g0n;
      st->k = 0;
      st->iters = iters;
      st->hcount = 0;
      st->hhead = 0;
      st->status = status;
      st->degen = 0;  // the flag reports accepted iterates only
      st->cur = 0;
      for (int i = 0; i < kHistory; ++i) st->rho[i] = st->aco[i] = (S)0;
      st->cvol[0] = cvol.x;
      st->cvol[1] = cvol.y;
      st->cvol[2] = cvol.z;
    }
    __syncwarp();
    if (iters == 0) {
      split_finalize<S>(ty, P, w, st, w.U, w.G, cell, 0, x, v, lane);
      continue;
    }
    if (lane == 0) P.act_out[atomicAdd(P.act_count_out, 1)] = item;
    // the history is empty here, so the first half of the two-loop recursion is Q = g
    NPFEM_PHASE_BEGIN(t_loop1)
    for (int e = lane; e < len; e += 32) w.Q[e] = w.G[e];
    __syncwarp();
    NPFEM_PHASE_END(t_loop1, kPhTwoLoop, P, lane)
  }
}

// Vector placement of the solve kernel: kZWorkspace (each cell's [n+1][3] vector in its
// workspace), kZShared ([n+1][3] per cell in shared memory) or kZSharedPerCoord ([n+1]
// per cell in shared memory, the three coordinates swept one after another).
constexpr int kZWorkspace = 0, kZShared = 1, kZSharedPerCoord = 2;

template <typename S, int kCells, int kPlace>
__device__ __forceinline__ void solve_group(const DevTypeView<S>& ty, const StepParams& P, char* const* base,
                                            double* zsm, int lane) {
  constexpr int zc = kPlace == kZSharedPerCoord ? 1 : 3;
  double* z[kCells];
  S* q[kCells];
#pragma unroll
  for (int c = 0; c < kCells; ++c) {
    CellWs<S> w = split_ws<S>(base[c], ty);
    z[c] = kPlace == kZWorkspace ? w.z : zsm + (size_t)c * zc * (ty.n + 1);
    q[c] = w.Q;
  }
  global_solve_n<S, kCells, true>(ty, z, kPlace != kZWorkspace, q, q, lane, kPlace == kZSharedPerCoord);
}

// Q <- A^-1 Q for every cell still iterating (the compacted list of iteration i).  A
// warp claims kCells list entries at a time and sweeps them together, so each factor
// entry it loads serves 3 x kCells right-hand sides; a short last group goes cell by
// cell.  One instantiation per cell count and vector placement keeps a single sweep
// variant (and its register allocation) per kernel.
template <typename S, int kCells, int kPlace>
__global__ void __launch_bounds__(128) npfem_k_solve(DevTypeView<S> ty, StepParams P) {
  extern __shared__ double smem_z[];
  constexpr int zc = kPlace == kZSharedPerCoord ? 1 : 3;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  double* zsm = smem_z + (size_t)wib * kCells * zc * (ty.n + 1);
  const int total = *P.act_count_in;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(P.queue_counter, kCells);
    item = __shfl_sync(kFull, item, 0);
    if (item >= total) break;
    char* base[kCells];
    const int cnt = total - item < kCells ? total - item : kCells;
#pragma unroll
    for (int c = 0; c < kCells; ++c)
      base[c] = P.scratch + (size_t)P.act_in[c < cnt ? item + c : item] * P.slot_bytes;
    NPFEM_PHASE_BEGIN(t_solve)
    if (cnt == kCells) {
      solve_group<S, kCells, kPlace>(ty, P, base, zsm, lane);
    } else {
      for (int c = 0; c < cnt; ++c) solve_group<S, 1, kPlace>(ty, P, base + c, zsm, lane);
    }
    NPFEM_PHASE_END(t_solve, kPhSolve, P, lane)
  }
}

// One sweep of a CTA of W warps over a level packing (Eqs. (7)-(8), as in chunk_sweep_n
// but cooperative): warp w applies sub-chunk w of every level to the shared vectors of
// the CTA's kCells cells ([n+1][3] doubles each, zstride bytes apart, the first at zs),
// with a barrier of the CTA before every level that touches a row written since the last
// barrier; the levels in between commute.  Each factor entry loaded updates every cell,
// and each cell sees its updates in the order of the one-cell sweep.
// Levels of the factor stream a warp of the CTA-cooperative sweep keeps in flight.
constexpr int kCtaPrefetch = 6;

template <int W, int kCells>
__device__ __forceinline__ void cta_sweep(int nlev, const int32_t* __restrict__ meta, const uint32_t* __restrict__ rc,
                                          const double* __restrict__ val, uint32_t zs, uint32_t zstride, int n,
                                          int warp, int lane) {
  int mb[kCtaPrefetch];
  uint32_t eb[kCtaPrefetch];
  double vb[kCtaPrefetch];
#pragma unroll
  for (int k = 0; k < kCtaPrefetch; ++k) {
    if (k < nlev) {
      const size_t sc = (size_t)k * W + warp;
      mb[k] = __ldg(meta + sc);
      eb[k] = __ldg(rc + sc * kChunk + lane);
      vb[k] = __ldg(val + sc * kChunk + lane);
    } else {
      mb[k] = 2;
      eb[k] = (uint32_t)n | ((uint32_t)n << 16);
      vb[k] = 0.0;
    }
  }
  for (int base = 0; base < nlev; base += kCtaPrefetch) {
#pragma unroll
    for (int k = 0; k < kCtaPrefetch; ++k) {
      const int lv = base + k;
      if (lv < nlev) {
        const int m = mb[k];
        const uint32_t e = eb[k];
        const double l = vb[k];
        const int nx = lv + kCtaPrefetch;
        if (nx < nlev) {
          const size_t sc = (size_t)nx * W + warp;
          mb[k] = __ldg(meta + sc);
          eb[k] = __ldg(rc + sc * kChunk + lane);
          vb[k] = __ldg(val + sc * kChunk + lane);
        }
        if (m & 1) __syncthreads();
        if (!(m & 2)) {
          const int r = (int)(e & 0xffffu), j = (int)(e >> 16);
          double xj[kCells][3], zr[kCells][3];
#pragma unroll
          for (int c = 0; c < kCells; ++c) {
            const uint32_t aj = zs + c * zstride + 24u * (uint32_t)j;
#pragma unroll
            for (int d = 0; d < 3; ++d) xj[c][d] = lds_f64(aj + 8 * d);
          }
#pragma unroll
          for (int c = 0; c < kCells; ++c) {
            const uint32_t ar = zs + c * zstride + 24u * (uint32_t)r;
#pragma unroll
            for (int d = 0; d < 3; ++d) zr[c][d] = fma(-l, xj[c][d], lds_f64(ar + 8 * d));
          }
#pragma unroll
          for (int c = 0; c < kCells; ++c) {
            const uint32_t ar = zs + c * zstride + 24u * (uint32_t)r;
#pragma unroll
            for (int d = 0; d < 3; ++d) sts_f64(ar + 8 * d, zr[c][d]);
          }
        }
      }
    }
  }
  __syncthreads();
}

// Index of the level packing for a CTA of W warps.
template <int W>
struct CtaPack {
  static constexpr int value = W == kCtaWarps[0] ? 0 : W == kCtaWarps[1] ? 1 : W == kCtaWarps[2] ? 2 : 3;
  static_assert(W == kCtaWarps[value], "no level packing for this CTA width");
};

// Resident CTAs per SM the CTA-cooperative solve is compiled for (a register budget of
// 65536 / (32 W x min_blocks) per thread).  One cell per CTA: the 2-warp CTA of the
// 642-vertex type holds a 15.4 KB vector, so shared memory admits 13 per SM, and 72
// registers let registers admit as many (at 96 registers only 10 fit); the wider CTAs
// keep the residency their shared memory allows for the larger types (6 or 8 warps: three
// 61.5 KB vectors of a 2562-vertex cell).  Two cells per CTA: shared memory admits 7
// 2-warp CTAs of the 642-vertex type (2 x 15.4 KB each).
template <int W, int kCells>
struct SolveCtaOccupancy {
  static constexpr int min_blocks =
      kCells == 1 ? (W == 2 ? 13 : (W == 4 ? 5 : 3)) : (W == 2 ? 7 : (W == 4 ? 4 : 1));
};

// Q <- A^-1 Q, one CTA of W warps per kCells cells at a time, for cells whose FP64 solve
// vectors ([n+1][3], 24(n+1) bytes each) are too large to keep one per warp in shared
// memory: the CTA's warps share the vectors and sweep the W-warp level packing of the
// factor together (Eqs. (7)-(8): permute, unit-lower forward sweep, D^-1, unit-upper
// backward sweep).  One cell per CTA: cells in batch order, ended ones skipped.  Two
// cells per CTA: pairs of the compacted list of cells still iterating (a last odd cell
// alone); each cell's arithmetic is that of the one-cell kernel.
template <typename S, int W, int kCells>
__global__ void __launch_bounds__(32 * W, (SolveCtaOccupancy<W, kCells>::min_blocks)) npfem_k_solve_cta(
    DevTypeView<S> ty, StepParams P) {
  constexpr int pk = CtaPack<W>::value;
  extern __shared__ double smem_z[];
  __shared__ int s_item;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = ty.n;
  const uint32_t zs = (uint32_t)__cvta_generic_to_shared(smem_z);
  const size_t zlen = 3 * ((size_t)n + 1);
  const uint32_t zstride = (uint32_t)(sizeof(double) * zlen);
  const int total = kCells == 1 ? P.ncells_list : *P.act_count_in;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(P.queue_counter, kCells);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= total) break;
    S* Q[kCells];
    int cnt = 1;
    if (kCells == 1) {
      char* base = P.scratch + (size_t)item * P.slot_bytes;
      const CellState<S>* cs = reinterpret_cast<const CellState<S>*>(base);
      if (cs->k >= cs->iters) continue;  // same header for the whole CTA: a uniform branch
      Q[0] = split_ws<S>(base, ty).Q;
    } else {
      cnt = total - item < kCells ? total - item : kCells;
#pragma unroll
      for (int c = 0; c < kCells; ++c)
        Q[c] = split_ws<S>(P.scratch + (size_t)P.act_in[c < cnt ? item + c : item] * P.slot_bytes, ty).Q;
    }
    NPFEM_PHASE_BEGIN(t_solve)
    for (int r = tid; r < n; r += 32 * W) {
      const int v = __ldg(&ty.perm[r]);
#pragma unroll
      for (int c = 0; c < kCells; ++c) {
        if (c < cnt) {
          const S q0 = Q[c][3 * v], q1 = Q[c][3 * v + 1], q2 = Q[c][3 * v + 2];
          smem_z[c * zlen + 3 * r] = (double)q0;
          smem_z[c * zlen + 3 * r + 1] = (double)q1;
          smem_z[c * zlen + 3 * r + 2] = (double)q2;
        }
      }
    }
    if (tid < 3)
#pragma unroll
      for (int c = 0; c < kCells; ++c) smem_z[c * zlen + 3 * n + tid] = 0.0;
    __syncthreads();
    if (cnt == kCells)
      cta_sweep<W, kCells>(ty.cta_nlev_fwd[pk], ty.cta_fwd_meta[pk], ty.cta_fwd_rc[pk], ty.cta_fwd_val[pk], zs,
                           zstride, n, warp, lane);
    else
      cta_sweep<W, 1>(ty.cta_nlev_fwd[pk], ty.cta_fwd_meta[pk], ty.cta_fwd_rc[pk], ty.cta_fwd_val[pk], zs, zstride,
                      n, warp, lane);
    for (int r = tid; r < n; r += 32 * W) {
      const double d = __ldg(&ty.dinv[r]);
#pragma unroll
      for (int c = 0; c < kCells; ++c) {
        smem_z[c * zlen + 3 * r] *= d;
        smem_z[c * zlen + 3 * r + 1] *= d;
        smem_z[c * zlen + 3 * r + 2] *= d;
      }
    }
    __syncthreads();
    if (cnt == kCells)
      cta_sweep<W, kCells>(ty.cta_nlev_bwd[pk], ty.cta_bwd_meta[pk], ty.cta_bwd_rc[pk], ty.cta_bwd_val[pk], zs,
                           zstride, n, warp, lane);
    else
      cta_sweep<W, 1>(ty.cta_nlev_bwd[pk], ty.cta_bwd_meta[pk], ty.cta_bwd_rc[pk], ty.cta_bwd_val[pk], zs, zstride,
                      n, warp, lane);
    for (int r = tid; r < n; r += 32 * W) {
      const int v = __ldg(&ty.perm[r]);
#pragma unroll
      for (int c = 0; c < kCells; ++c) {
        if (c < cnt) {
          Q[c][3 * v] = (S)smem_z[c * zlen + 3 * r];
          Q[c][3 * v + 1] = (S)smem_z[c * zlen + 3 * r + 1];
          Q[c][3 * v + 2] = (S)smem_z[c * zlen + 3 * r + 2];
        }
      }
    }
    NPFEM_PHASE_END(t_solve, kPhSolve, P, warp == 0 ? lane : 1)
    __syncthreads();
  }
}

template <typename S, bool kLim>
__global__ void __launch_bounds__(128, IterOccupancy<S>::min_blocks) npfem_k_iter(DevTypeView<S> ty, StepParams P, S* x, S* v) {
  const int lane = threadIdx.x & 31;
  const int n = ty.n, len = 3 * n;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(P.queue_counter, 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= P.ncells_list) break;
    const int cell = P.cell_list[item];
    char* base = P.scratch + (size_t)item * P.slot_bytes;
    CellState<S>* st = reinterpret_cast<CellState<S>*>(base);
    const int k = st->k, iters = st->iters;
    if (k >= iters) continue;
    CellWs<S> w = split_ws<S>(base, ty);
    S* U = st->cur ? w.UT : w.U;
    S* UT = st->cur ? w.U : w.UT;
    S* G = st->cur ? w.GT : w.G;
    S* GT = st->cur ? w.G : w.GT;
    const V3<S> cvol{st->cvol[0], st->cvol[1], st->cvol[2]};
    const double fx = st->fx;
    int hcount = st->hcount, hhead = st->hhead;
    NPFEM_PHASE_BEGIN(t_loop2)
    // Second half, oldest -> newest pairs, fused like the first: each pass applies one
    // pair's update and accumulates the next pair's y . Q; the last pass writes D = -Q
    // and accumulates g . D (Q's final value is not kept: the fallback below and the next
    // first half overwrite it).
    double gd;
    {
      Acc<S> agd;
      if (hcount == 0) {
        for (int e = lane; e < len; e += 32) {
          const S d = -w.Q[e];
          w.D[e] = d;
          agd.add_prod(G[e], d);
        }
      } else {
        int i = (hhead - hcount + kHistory) % kHistory;
        S acc = 0;
        {
          const S* yi = w.hy + (size_t)i * len;
          for (int e = lane; e < len; e += 32) acc += yi[e] * w.Q[e];
        }
        for (int q = hcount - 1; q >= 0; --q) {
          const S b = st->rho[i] * warp_sum<S>(acc);
          const S c = st->aco[i] - b;
          const S* si = w.hs + (size_t)i * len;
          if (q > 0) {
            const int inext = (hhead - 1 - (q - 1) + kHistory) % kHistory;
            acc = update_dot<S>(w.Q, c, si, w.hy + (size_t)inext * len, len, lane);
            i = inext;
          } else {
            update_negate<S>(w.Q, c, si, G, w.D, agd, len, lane);
          }
        }
      }
      gd = agd.total();
    }
    NPFEM_PHASE_END(t_loop2, kPhTwoLoop, P, lane)
    if (!(gd < 0.0)) {  // not a descent direction: drop history, plain PD step
      hcount = 0;
      hhead = 0;
      global_solve<S>(ty, w.z, false, G, w.Q, lane, false);
      for (int e = lane; e < len; e += 32) w.D[e] = -w.Q[e];
      __syncwarp();
      gd = vdot64<S>(G, w.D, len, lane);
    }
    double alpha = 1.0, ft = 0.0;
    bool degen = false;
    int status = 0;
    for (int h = 0; h <= kMaxHalvings; ++h) {
      const S sa = (S)alpha;
      for (int e = lane; e < len; e += 32) UT[e] = U[e] + sa * w.D[e];
      __syncwarp();
      NPFEM_PHASE_BEGIN(t_obj)
      EvalOut et = eval_objective<S, kLim ? 1 : 0>(ty, P, w, UT, GT, cvol, cell, lane);
      NPFEM_PHASE_END(t_obj, kPhObjective, P, lane)
      ft = et.energy;
      degen = et.degenerate;  // the trial that ends the search is the accepted one
      double gtd = vdot64<S>(GT, w.D, len, lane);
      bool armijo = ft <= fx + kArmijoC1 * alpha * gd;
      bool approx = (gtd <= (2.0 * kArmijoC1 - 1.0) * gd) && (ft <= fx + kEnergyGuardEps * fabs(fx));
      if (armijo || approx) break;
      if (h == kMaxHalvings) {
        status |= 1;
        break;
      }
      alpha *= 0.5;
    }
    // converged-residual mode: the accepted trial ends the step when |g| < tol |g0|
    const bool stop = P.tol > 0.0 && sqrt(vdot64<S>(GT, GT, len, lane)) < P.tol * st->g0n;
    NPFEM_PHASE_BEGIN(t_hist)
    S new_rho = (S)0;
    bool keep = false;
    if (k < iters - 1 && !stop) {
      S* si = w.hs + (size_t)hhead * len;
      S* yi = w.hy + (size_t)hhead * len;
      Acc<S> asy, ass, ayy;
      for (int e = lane; e < len; e += 32) {
        S s = UT[e] - U[e];
        S y = GT[e] - G[e];
        si[e] = s;
        yi[e] = y;
        asy.add_prod(s, y);
        ass.add_prod(s, s);
        ayy.add_prod(y, y);
      }
      const double sy = asy.total(), ss = ass.total(), yy = ayy.total();
      if (sy > kCurvatureEps * sqrt(ss) * sqrt(yy)) {
        keep = true;
        new_rho = (S)(1.0 / sy);
      }
      __syncwarp();
    }
    NPFEM_PHASE_END(t_hist, kPhHistory, P, lane)
    if (P.alpha_log && k < P.alpha_log_len && lane == 0) P.alpha_log[(size_t)cell * P.alpha_log_len + k] = alpha;
    if (lane == 0) {
      if (keep) {
        st->rho[hhead] = new_rho;
        hhead = (hhead + 1) % kHistory;
        hcount = hcount < kHistory ? hcount + 1 : kHistory;
      }
      st->hcount = hcount;
      st->hhead = hhead;
      st->fx = ft;
      st->cur ^= 1;
      st->k = k + 1;
      st->status |= status;
      if (degen) st->degen = 1;
    }
    __syncwarp();
    // the accepted trial (UT, GT) is the new current iterate
    if (k + 1 < iters && !stop) {
      if (lane == 0) P.act_out[atomicAdd(P.act_count_out, 1)] = item;
      NPFEM_PHASE_BEGIN(t_loop1)
      two_loop_first<S>(w, st, GT, len, lane);
      NPFEM_PHASE_END(t_loop1, kPhTwoLoop, P, lane)
    } else {
      split_finalize<S>(ty, P, w, st, UT, GT, cell, k + 1, x, v, lane);
    }
  }
}

}  // namespace npfem
