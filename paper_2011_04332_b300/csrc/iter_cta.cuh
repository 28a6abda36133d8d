// CTA-cooperative iteration kernels of the split step (k_begin_cta, k_iter_cta): one CTA
// of W warps advances one cell at a time, through the same steps as k_begin and k_iter
// (K1 prediction, K2 objective and gradient, K3 two-loop recursion around the FP64 solve
// of k_solve, K5 line search, K6 history, K7 write-back).
//
// During every objective evaluation the cell's start positions X, its trial displacement
// U and its gradient G live in shared memory.  Triangles and hinges are visited colour by
// colour (the host stores them so that no two elements of a colour share a vertex), so
// each colour adds its gradient contributions to G in place: no atomics, no per-element
// records in global memory and no per-vertex gather through them, and the order of the
// additions is fixed.  Element arithmetic is that of the warp kernels (triangle_terms,
// hinge_terms); sums run in another order, so the two agree to rounding.  Reductions over
// the cell are CTA-wide and depend on the CTA width, which the library fixes per cell
// type (it is not a tuning parameter), so a cell's result does not depend on the launch.
#pragma once
#include "split_kernels.cuh"

namespace npfem {

constexpr int kIterCtaMaxWarps = 16;

// Resident 512-thread CTAs the CTA iteration kernels are compiled for: a register budget
// of 64 per thread for the FP32 form and 128 for FP64, those of the warp kernels.
template <typename S>
struct IterCtaOccupancy {
  static constexpr int min_blocks = 1;
};
template <>
struct IterCtaOccupancy<float> {
  static constexpr int min_blocks = 2;
};

// Shared scratch of a CTA: double-buffered per-warp partial sums (one barrier per
// reduction: a buffer is written again only two reductions later, when every thread has
// passed the barrier of the reduction in between), in FP64 and in FP32 (the FP32 form's
// two-loop dot products), the work-queue item, and the scalars that one warp derives
// from a reduction for the whole CTA (published by a later barrier: the area and volume
// terms of an evaluation, the curvature test of a history pair).
struct CtaShared {
  double red[2][kIterCtaMaxWarps * 4];
  float redf[2][kIterCtaMaxWarps];
  double e_av;     // area + volume energy of the evaluation
  double kA, kV;   // their gradient coefficients
  int keep;        // the new history pair passed the curvature test
  int item;
};

// The working-precision partial-sum buffer of cta_sum_s.
template <typename S>
__device__ __forceinline__ S* sum_buffer(CtaShared& sh, int par);
template <>
__device__ __forceinline__ float* sum_buffer<float>(CtaShared& sh, int par) {
  return sh.redf[par];
}
template <>
__device__ __forceinline__ double* sum_buffer<double>(CtaShared& sh, int par) {
  return sh.red[par];
}

// Sums over the CTA of K <= 4 per-thread FP64 values; every thread receives the totals.
// The FP64 pipe is the scarce unit (a warp-wide FP64 add occupies it for 64 cycles
// whatever the active lanes), so the lanes reduce-scatter: at the first log2(K4) shuffle
// steps (K4 = K rounded up to a power of two) each lane keeps half of the values it still
// carries, so every later step is a single add for all values at once; lane l ends with
// value l mod K4 summed over the warp.  The warp totals go to shared memory, and after
// the barrier lane k*nw + q of every warp loads value k of warp q and a butterfly over the
// nw lanes of each value adds them (nw a power of two, 32 / nw values per round).  Every
// lane of every warp performs the same additions on the same operands, so all threads
// receive identical totals.  Call discipline: all threads of the CTA make the same
// sequence of calls (par alternates the buffers).
template <int K>
__device__ __forceinline__ void cta_sum(double (&v)[K], CtaShared& sh, int& par) {
  static_assert(K >= 1 && K <= 4, "cta_sum takes 1 to 4 values");
  constexpr int K4 = K == 1 ? 1 : (K == 2 ? 2 : 4);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double w[K4];
#pragma unroll
  for (int k = 0; k < K4; ++k) w[k] = k < K ? v[k] : 0.0;
  // reduce-scatter over the lane bits 4, 3 (K4 = 4) or 4 (K4 = 2): after it, a lane's
  // w[0] holds the partial sum of value (lane >> (5 - log2 K4)) over the lanes that share
  // its remaining bits
  if (K4 >= 2) {
    const bool hi = lane & 16;
#pragma unroll
    for (int k = 0; k < K4 / 2; ++k) {
      const double send = hi ? w[k] : w[k + K4 / 2];
      const double keep = hi ? w[k + K4 / 2] : w[k];
      w[k] = keep + __shfl_xor_sync(kFull, send, 16);
    }
  }
  if (K4 == 4) {
    const bool hi = lane & 8;
    const double send = hi ? w[0] : w[1];
    const double keep = hi ? w[1] : w[0];
    w[0] = keep + __shfl_xor_sync(kFull, send, 8);
  }
  double x = w[0];
#pragma unroll
  for (int o = (K4 == 4 ? 4 : (K4 == 2 ? 8 : 16)); o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  // lane l now holds value (l >> 3) (K4 = 4), (l >> 4) (K4 = 2) or the only value
  double* r = sh.red[par];
  par ^= 1;
  const int vid = K4 == 4 ? lane >> 3 : (K4 == 2 ? lane >> 4 : 0);
  if ((lane & (32 / K4 - 1)) == 0 && vid < K) r[vid * nw + warp] = x;
  __syncthreads();
  // 32 / nw values per round (nw a power of two): lane j*nw + q loads value kb + j of warp
  // q, and a butterfly over the nw lanes of each value adds the warps' totals
  const int per_round = 32 / nw;
  for (int kb = 0; kb < K; kb += per_round) {
    const int j = lane / nw, k0 = kb + j;
    double y = (j < per_round && k0 < K) ? r[k0 * nw + (lane % nw)] : 0.0;
    for (int o = nw >> 1; o > 0; o >>= 1) y += __shfl_xor_sync(kFull, y, o);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const double t = __shfl_sync(kFull, y, ((k - kb) & 31) * nw & 31);
      if (k >= kb && k < kb + per_round) v[k] = t;
    }
  }
}

__device__ __forceinline__ double cta_sum1(double x, CtaShared& sh, int& par) {
  double v[1] = {x};
  cta_sum<1>(v, sh, par);
  return v[0];
}

// Sum over the CTA in the working precision S, for the dot products of the two-loop
// recursion (FP32 in the FP32 form, like the warp kernels' warp sums): lanes by shuffles,
// then the warp totals in warp order, kept in S (no conversion through FP64).  Same call
// discipline as cta_sum (the FP32 buffers alternate with the same parity).
template <typename S>
__device__ __forceinline__ S cta_sum_s(S x, CtaShared& sh, int& par) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  x = warp_sum<S>(x);
  S* r = sum_buffer<S>(sh, par);
  par ^= 1;
  if (lane == 0) r[warp] = x;
  __syncthreads();
  S s = 0;
  for (int q = 0; q < nw; ++q) s += r[q];
  return s;
}

// Requests a global vector of len elements into L2 (one prefetch per 128-byte line,
// spread over the CTA's threads; the line of the last element too, for vectors that do
// not start on a line) ahead of the pass that reads it.  The two-loop passes are latency
// bound — each waits for its loads, then for its CTA-wide reduction — so the next pass's
// vectors come from DRAM while the current pass runs.
template <typename S>
__device__ __forceinline__ void prefetch_l2(const S* p, int len, int tid, int nt) {
  constexpr int kLine = 128 / (int)sizeof(S);
  for (int e = tid * kLine; e < len; e += nt * kLine) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + e));
  if (tid == 0 && len > 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + len - 1));
}

// Last pass of the second half of the two-loop recursion fused with the line search's
// first trial (step 1): d = -(q + c u), UT = Us = U + d; agd accumulates g . d.  Four
// elements per thread in flight, as in update_dot.
template <typename S>
__device__ __forceinline__ void cta_negate_trial(const S* q, S c, const S* u, const S* g, const S* U, S* d, S* UT,
                                                 S* Us, Acc<S>& agd, int len, int tid, int nt) {
  int e = tid;
  for (; e + 3 * nt < len; e += 4 * nt) {
    S qv[4], uv[4], gv[4], Uv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      qv[j] = q[e + nt * j];
      uv[j] = u[e + nt * j];
      gv[j] = g[e + nt * j];
      Uv[j] = U[e + nt * j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const S dv = -(qv[j] + c * uv[j]);
      d[e + nt * j] = dv;
      agd.add_prod(gv[j], dv);
      const S ut = Uv[j] + dv;
      UT[e + nt * j] = ut;
      Us[e + nt * j] = ut;
    }
  }
  for (; e < len; e += nt) {
    const S dv = -(q[e] + c * u[e]);
    d[e] = dv;
    agd.add_prod(g[e], dv);
    const S ut = U[e] + dv;
    UT[e] = ut;
    Us[e] = ut;
  }
}

// Elastic part of Rayleigh damping, (c_beta/dt)/2 U^T L U, element by element and colour
// by colour into the shared gradient G (the terms of damping_elastic).  Returns this
// thread's share of the damping energy.
template <typename S>
__device__ __noinline__ double damping_elastic_cta(const DevTypeView<S>& ty, S dl, const S* U, S* G, int tid,
                                                   int nt) {
  const S half = (S)0.5;
  double e = 0.0;
  for (int c = 0; c < ty.ntc; ++c) {
    const int lo = __ldg(&ty.tri_cptr[c]), hi = __ldg(&ty.tri_cptr[c + 1]);
    for (int t = lo + tid; t < hi; t += nt) {
      const int i0 = __ldg(&ty.tris[3 * t]), i1 = __ldg(&ty.tris[3 * t + 1]), i2 = __ldg(&ty.tris[3 * t + 2]);
      const V3<S> u0 = ld3(U, i0);
      const V3<S> u1 = ld3(U, i1) - u0, u2 = ld3(U, i2) - u0;
      const S d00 = __ldg(&ty.Dinv[3 * t]), d01 = __ldg(&ty.Dinv[3 * t + 1]), d11 = __ldg(&ty.Dinv[3 * t + 2]);
      const S wd = dl * __ldg(&ty.w_tri[t]);
      const V3<S> F0 = d00 * u1, F1 = d01 * u1 + d11 * u2;
      e += (double)(half * wd * (dot(F0, F0) + dot(F1, F1)));
      const V3<S> P0 = wd * F0, P1 = wd * F1;
      const V3<S> g1 = d00 * P0 + d01 * P1, g2 = d11 * P1;
      st3(G, i0, ld3(G, i0) - (g1 + g2));
      st3(G, i1, ld3(G, i1) + g1);
      st3(G, i2, ld3(G, i2) + g2);
    }
    __syncthreads();
  }
  for (int c = 0; c < ty.nhc; ++c) {
    const int lo = __ldg(&ty.hinge_cptr[c]), hi = __ldg(&ty.hinge_cptr[c + 1]);
    for (int h = lo + tid; h < hi; h += nt) {
      const int4 hv = ldg4(ty.hinges + 4 * h);
      const typename Q4Of<S>::type cv = ldg4(ty.c_hinge + 4 * h);
      const V3<S> ui = ld3(U, hv.x);
      const V3<S> KU = cv.y * (ld3(U, hv.y) - ui) + cv.z * (ld3(U, hv.z) - ui) + cv.w * (ld3(U, hv.w) - ui);
      const S wd = dl * __ldg(&ty.w_hinge[h]);
      e += (double)(half * wd * dot(KU, KU));
      const V3<S> r = wd * KU;
      st3(G, hv.x, ld3(G, hv.x) + cv.x * r);
      st3(G, hv.y, ld3(G, hv.y) + cv.y * r);
      st3(G, hv.z, ld3(G, hv.z) + cv.z * r);
      st3(G, hv.w, ld3(G, hv.w) + cv.w * r);
    }
    __syncthreads();
  }
  return e;
}

struct CtaEval {
  double energy;  // f(X + U)
  double gtd;     // G . D (D given), else 0
  double gg;      // G . G
  bool degenerate;
};

// f(X + U) and its gradient for one cell, by the CTA: Xs, Us in shared memory (complete
// and visible when called), the gradient assembled in the shared Gs and written to Gout
// (global); D optional (the search direction for G . D).  Passes: strain-limit matrices
// (limited types), area and volume (FP64 sums), inertia (and damping's mass part) into
// Gs, triangles and hinges colour by colour (and damping's elastic part), contact planes
// and box walls per vertex, then the write of Gout with the dot products.
template <typename S, int kLim>
__device__ CtaEval cta_objective(const DevTypeView<S>& ty, const StepParams& P, const CellWs<S>& w, const S* Xs,
                                 const S* Us, S* Gs, S* Gout, const S* D, V3<S> cvol, int cell, CtaShared& sh,
                                 int& par) {
  const int n = ty.n, T = ty.T, len = 3 * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool limited = kLim == 1 || (kLim == 2 && ty.limited);
  if (limited) strain_limit_pass<S>(ty, Xs, Us, w.corner, tid, nt);
  NPFEM_PHASE_BEGIN(t_area)
  Acc<S> a_sum, v_sum;
  for (int t = tid; t < T; t += nt) {
    const int4 tv = ldg4(ty.tri4 + 4 * t);
    const V3<S> e1 = edge(Xs, Us, tv.x, tv.y), e2 = edge(Xs, Us, tv.x, tv.z);
    const V3<S> N = cross(e1, e2);
    a_sum.add(sqrt(dot(N, N)));
    const V3<S> q0 = (ld3(Xs, tv.x) + ld3(Us, tv.x)) - cvol;
    v_sum.add(dot(q0, N));
  }
  double av[2] = {a_sum.part(), v_sum.part()};
  cta_sum<2>(av, sh, par);  // also publishes the strain-limit matrices of the pass above
  // The area and volume terms are scalar FP64 work on the totals; every FP64 warp
  // instruction occupies the FP64 pipe for the whole warp, so one warp derives them and
  // the barrier after the inertia pass publishes them.
  if (tid < 32) {
    const double A = 0.5 * av[0];
    const double V = av[1] * (1.0 / 6.0);
    const double dA = A - ty.A0, dV = V - ty.V0;
    if (tid == 0) {
      sh.e_av = 0.5 * ty.w_area * dA * dA * ty.inv_A0 + 0.5 * ty.w_vol * dV * dV * ty.inv_V0;
      sh.kA = ty.w_area * dA * ty.inv_A0;
      sh.kV = ty.w_vol * dV * ty.inv_V0;
    }
  }
  NPFEM_PHASE_END(t_area, kPhAreaVolume, P, tid)

  NPFEM_PHASE_BEGIN(t_acc)
  const S half = (S)0.5, idt2 = (S)ty.idt2;
  // The table rows of a thread's first element in the next colour class are loaded before
  // the barrier that ends the current class (or the inertia pass), so their L2 round trip
  // overlaps the wait; they are live only across the barrier, not through the element
  // arithmetic.
  int4 tv_next = make_int4(0, 0, 0, 0), hv_next = make_int4(0, 0, 0, 0);
  typename Q4Of<S>::type tc_next{}, cv_next{};
  S k0n_next = 0, wh_next = 0;
  auto load_tri = [&](int lo, int hi) {
    if (lo + tid < hi) {
      tv_next = ldg4(ty.tri4 + 4 * (lo + tid));
      tc_next = ldg4(ty.trc + 4 * (lo + tid));
    }
  };
  auto load_hinge = [&](int lo, int hi) {
    if (lo + tid < hi) {
      hv_next = ldg4(ty.hinges + 4 * (lo + tid));
      cv_next = ldg4(ty.c_hinge + 4 * (lo + tid));
      k0n_next = __ldg(&ty.K0[4 * (lo + tid) + 3]);
      wh_next = __ldg(&ty.w_hinge[lo + tid]);
    }
  };
  if (ty.ntc > 0)
    load_tri(__ldg(&ty.tri_cptr[0]), __ldg(&ty.tri_cptr[1]));
  else if (ty.nhc > 0)
    load_hinge(__ldg(&ty.hinge_cptr[0]), __ldg(&ty.hinge_cptr[1]));
  Acc<S> e_el;
  for (int v = tid; v < n; v += nt) {
    const V3<S> du = ld3(Us, v) - ld3(w.W, v);
    const S m = __ldg(&ty.mass[v]);
    e_el.add(half * m * idt2 * dot(du, du));
    st3(Gs, v, (m * idt2) * du);
  }
  // damping's mass part visits the same vertices per thread: no barrier in between
  if (ty.damp_m != 0.0) e_el.add((S)damping_mass<S>(ty.mass, n, (S)ty.damp_m, Us, Gs, tid, nt));
  __syncthreads();  // also publishes the area and volume terms
  const S kA = (S)sh.kA, kV = (S)sh.kV;
  bool degen = false;
  auto triangle = [&](int t, const int4& tv, const typename Q4Of<S>::type& tc) {
    const int i0 = tv.x, i1 = tv.y, i2 = tv.z;
    const V3<S> e1 = edge(Xs, Us, i0, i1), e2 = edge(Xs, Us, i0, i2);
    const V3<S> q0 = (ld3(Xs, i0) + ld3(Us, i0)) - cvol;
    V3<S> g0, g1, g2;
    triangle_terms<S>(e1, e2, q0, tc, limited ? w.corner + 9 * t : nullptr, kA, kV, e_el, degen, g0, g1, g2);
    st3(Gs, i0, ld3(Gs, i0) + g0);
    st3(Gs, i1, ld3(Gs, i1) + g1);
    st3(Gs, i2, ld3(Gs, i2) + g2);
  };
  for (int c = 0; c < ty.ntc; ++c) {
    const int lo = __ldg(&ty.tri_cptr[c]), hi = __ldg(&ty.tri_cptr[c + 1]);
    if (lo + tid < hi) {
      triangle(lo + tid, tv_next, tc_next);
      for (int t = lo + tid + nt; t < hi; t += nt) triangle(t, ldg4(ty.tri4 + 4 * t), ldg4(ty.trc + 4 * t));
    }
    if (c + 1 < ty.ntc)
      load_tri(hi, __ldg(&ty.tri_cptr[c + 2]));
    else if (ty.nhc > 0)
      load_hinge(__ldg(&ty.hinge_cptr[0]), __ldg(&ty.hinge_cptr[1]));
    __syncthreads();
  }
  auto hinge = [&](int h, const int4& hv, const typename Q4Of<S>::type& cv, S k0n, S wh) {
    const V3<S> K = hinge_vector<S>(Xs, Us, hv, cv);
    // the bending term of hinge_terms, with |K0| and w_e given
    const S kn = sqrt(dot(K, K));
    V3<S> p;
    if (kn < (S)kDegenerateNorm) {
      p = {__ldg(&ty.K0[4 * h]), __ldg(&ty.K0[4 * h + 1]), __ldg(&ty.K0[4 * h + 2])};
    } else {
      p = (k0n / kn) * K;
    }
    const V3<S> d = K - p;
    e_el.add((S)0.5 * wh * dot(d, d));
    const V3<S> r = wh * d;
    st3(Gs, hv.x, ld3(Gs, hv.x) + cv.x * r);
    st3(Gs, hv.y, ld3(Gs, hv.y) + cv.y * r);
    st3(Gs, hv.z, ld3(Gs, hv.z) + cv.z * r);
    st3(Gs, hv.w, ld3(Gs, hv.w) + cv.w * r);
  };
  for (int c = 0; c < ty.nhc; ++c) {
    const int lo = __ldg(&ty.hinge_cptr[c]), hi = __ldg(&ty.hinge_cptr[c + 1]);
    if (lo + tid < hi) {
      hinge(lo + tid, hv_next, cv_next, k0n_next, wh_next);
      for (int h = lo + tid + nt; h < hi; h += nt)
        hinge(h, ldg4(ty.hinges + 4 * h), ldg4(ty.c_hinge + 4 * h), __ldg(&ty.K0[4 * h + 3]), __ldg(&ty.w_hinge[h]));
    }
    if (c + 1 < ty.nhc) load_hinge(hi, __ldg(&ty.hinge_cptr[c + 2]));
    __syncthreads();
  }
  if (ty.damp_l != 0.0) e_el.add((S)damping_elastic_cta<S>(ty, (S)ty.damp_l, Us, Gs, tid, nt));
  double e_ct = 0.0;
  if (P.contact_count) {
    // contact planes of the step, (w/2) max(0, delta - gap)^2 each, then the box walls
    const int64_t off = P.offsets[cell];
    for (int v = tid; v < n; v += nt) {
      const int nc = P.contact_count[off + v];
      if (nc == 0) continue;
      V3<S> g = ld3(Gs, v);
      const V3<S> p = ld3(Xs, v) + ld3(Us, v);
      for (int m = 0; m < nc; ++m) {
        const double* pl = P.contact_plane + 8 * (off + v) + 4 * m;
        const double gap = pl[0] * (double)p.x + pl[1] * (double)p.y + pl[2] * (double)p.z - pl[3];
        const double pen = P.contact_delta - gap;
        if (pen > 0.0) {
          e_ct += 0.5 * P.contact_weight * pen * pen;
          const double fw = -P.contact_weight * pen;
          g.x += (S)(fw * pl[0]);
          g.y += (S)(fw * pl[1]);
          g.z += (S)(fw * pl[2]);
        }
      }
      st3(Gs, v, g);
    }
    if (P.box)
      e_ct += wall_pass<S>(static_cast<const S*>(P.x_state), off, P.n_total, P.contact_delta, P.contact_weight,
                           P.box, Xs, Us, Gs, n, tid, nt);
    __syncthreads();  // the write below visits the gradient by component, not by vertex
  }
  Acc<S> agtd, agg;
  for (int e = tid; e < len; e += nt) {
    const S g = Gs[e];
    Gout[e] = g;
    if (D) agtd.add_prod(g, D[e]);
    agg.add_prod(g, g);
  }
  double r[3] = {e_el.part() + e_ct, agtd.part(), agg.part()};
  const bool any_degen = __syncthreads_or(degen);
  cta_sum<3>(r, sh, par);
  NPFEM_PHASE_END(t_acc, kPhGather, P, tid)
  CtaEval o;
  o.energy = r[0] + sh.e_av;
  o.gtd = r[1];
  o.gg = r[2];
  o.degenerate = any_degen;
  return o;
}

// First half of the two-loop recursion by the CTA: Q = g, newest -> oldest pairs (the
// pass structure of two_loop_first, with CTA-wide dot products), run in place on the shared
// gradient Gs (not needed afterwards): the vector stays on chip through the passes and the
// last pass writes Q to the workspace for the solve.  Every thread updates only its own
// elements (e = tid + k nt in every pass), so the passes need no barrier of their own.
// newest_dot: when non-null, this thread's partial sum of s . g for the newest pair,
// already accumulated (in the same order) by the history update that wrote the pair.
template <typename S>
__device__ __forceinline__ void cta_two_loop_first(const CellWs<S>& w, CellState<S>* st, int hc, int hh, S* Gs,
                                                   int len, CtaShared& sh, int& par, const S* newest_dot) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (hc == 0) {
    for (int e = tid; e < len; e += nt) w.Q[e] = Gs[e];
    return;
  }
  int i = (hh - 1 + kHistory) % kHistory;
  if (hc > 1) prefetch_l2(w.hs + (size_t)((hh - 2 + kHistory) % kHistory) * len, len, tid, nt);
  S acc = 0;
  if (newest_dot) {
    acc = *newest_dot;
  } else {
    const S* si = w.hs + (size_t)i * len;
    for (int e = tid; e < len; e += nt) acc += si[e] * Gs[e];
  }
  for (int q = 0; q < hc; ++q) {
    // the pass of pair q (newest first) reads y_q and s_{q+1}; fetch the next pass's
    if (q + 1 < hc) {
      prefetch_l2(w.hy + (size_t)((hh - 1 - (q + 1) + kHistory) % kHistory) * len, len, tid, nt);
      if (q + 2 < hc) prefetch_l2(w.hs + (size_t)((hh - 1 - (q + 2) + kHistory) % kHistory) * len, len, tid, nt);
    }
    const S a = st->rho[i] * cta_sum_s<S>(acc, sh, par);
    if (tid == 0) st->aco[i] = a;
    const S* yi = w.hy + (size_t)i * len;
    if (q + 1 < hc) {
      const int inext = (hh - 1 - (q + 1) + kHistory) % kHistory;
      acc = update_dot<S>(Gs, -a, yi, w.hs + (size_t)inext * len, len, tid, nt);
      i = inext;
    } else {
      for (int e = tid; e < len; e += nt) w.Q[e] = Gs[e] - a * yi[e];
    }
  }
}

// a + (X + U) rounded once to S: exactly in FP64 for S = double; for S = float by a
// compensated FP32 sum (the rounding errors of X + U and of a + (X + U), each recovered
// exactly by Knuth's TwoSum, added back at the end), which equals the FP64 sum rounded to
// FP32 but for rare double-rounding ties and leaves the FP64 pipe to the solves.
__device__ __forceinline__ double anchored_sum(double a, double X, double U) { return a + (X + U); }
__device__ __forceinline__ float anchored_sum(float a, float X, float U) {
  const float s = X + U, bs = s - X;
  const float e1 = (X - (s - bs)) + (U - bs);
  const float t = a + s, bt = t - a;
  const float e2 = (a - (t - bt)) + (s - bt);
  return t + (e1 + e2);
}

// K7 by the CTA: x_{n+1} = anchor + X + U, v_{n+1} = U / dt, residual |g| / |g0|, status.
template <typename S>
__device__ void cta_finalize(const DevTypeView<S>& ty, const StepParams& P, CellState<S>* st, const S* Xs,
                             const S* Us, double gg, int cell, int done, S* x, S* v) {
  const int n = ty.n, tid = threadIdx.x, nt = blockDim.x;
  const int64_t off = P.offsets[cell], Nt = P.n_total;
  NPFEM_PHASE_BEGIN(t_write)
  const S ax = x[off], ay = x[Nt + off], az = x[2 * Nt + off];
  const S idt = (S)ty.inv_dt;
  bool bad = false;
  for (int k = tid; k < n; k += nt) {
    const S nx = anchored_sum(ax, Xs[3 * k], Us[3 * k]);
    const S ny = anchored_sum(ay, Xs[3 * k + 1], Us[3 * k + 1]);
    const S nz = anchored_sum(az, Xs[3 * k + 2], Us[3 * k + 2]);
    const S vx = Us[3 * k] * idt, vy = Us[3 * k + 1] * idt, vz = Us[3 * k + 2] * idt;
    bad = bad || !isfinite(nx) || !isfinite(ny) || !isfinite(nz) || !isfinite(vx) || !isfinite(vy) ||
          !isfinite(vz);
    if (k != 0) {
      x[off + k] = nx;
      x[Nt + off + k] = ny;
      x[2 * Nt + off + k] = nz;
    }
    v[off + k] = vx;
    v[Nt + off + k] = vy;
    v[2 * Nt + off + k] = vz;
  }
  // vertex 0 is the anchor: every thread read it above, so it is written after the barrier
  bad = __syncthreads_or(bad);
  if (tid == 0) {
    x[off] = anchored_sum(ax, Xs[0], Us[0]);
    x[Nt + off] = anchored_sum(ay, Xs[1], Us[1]);
    x[2 * Nt + off] = anchored_sum(az, Xs[2], Us[2]);
    int status = st->status;
    if (st->degen) status |= 2;
    if (bad) status |= 4;
    if (P.status_out) P.status_out[cell] = status;
    if (P.residual_out) P.residual_out[cell] = st->g0n > 0.0 ? sqrt(gg) / st->g0n : 0.0;
    if (P.iters_done) P.iters_done[cell] = done;
    st->k = st->iters;
  }
  NPFEM_PHASE_END(t_write, kPhWrite, P, tid)
}

// Shared-memory arrays of the CTA iteration kernels: X, U and G of one cell.
template <typename S>
__host__ __device__ constexpr size_t iter_cta_smem_bytes(int n) {
  return sizeof(S) * 9 * (size_t)n;
}

// K1 and the first objective evaluation of every cell of the list, one cell per CTA at a
// time (work queue): X = x_n - anchor, W = U = dt v_n + dt^2 M^-1 f, the centre of X, f
// and g at U, the state header, then Q = g (the history is empty) or, with no iterations,
// the write-back.
template <typename S, bool kLim>
__global__ void __launch_bounds__(32 * kIterCtaMaxWarps, IterCtaOccupancy<S>::min_blocks)
    npfem_k_begin_cta(DevTypeView<S> ty, StepParams P, int max_iters, S* x, S* v, const S* f) {
  extern __shared__ __align__(16) unsigned char cta_smem[];
  __shared__ CtaShared sh;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n = ty.n, len = 3 * n;
  S* Xs = reinterpret_cast<S*>(cta_smem);
  S* Us = Xs + len;
  S* Gs = Us + len;
  int par = 0;
  for (;;) {
    if (tid == 0) sh.item = atomicAdd(P.queue_counter, 1);
    __syncthreads();
    const int item = sh.item;
    __syncthreads();
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
    for (int k = tid; k < n; k += nt) {
      const S px = x[off + k] - ax, py = x[Nt + off + k] - ay, pz = x[2 * Nt + off + k] - az;
      w.X[3 * k] = px;
      w.X[3 * k + 1] = py;
      w.X[3 * k + 2] = pz;
      Xs[3 * k] = px;
      Xs[3 * k + 1] = py;
      Xs[3 * k + 2] = pz;
      cx.add(px);
      cy.add(py);
      cz.add(pz);
      const S im = __ldg(&ty.inv_mass[k]);
      const S wx = sdt * v[off + k] + sdt2 * f[off + k] * im;
      const S wy = sdt * v[Nt + off + k] + sdt2 * f[Nt + off + k] * im;
      const S wz = sdt * v[2 * Nt + off + k] + sdt2 * f[2 * Nt + off + k] * im;
      w.W[3 * k] = wx;
      w.W[3 * k + 1] = wy;
      w.W[3 * k + 2] = wz;
      w.U[3 * k] = wx;
      w.U[3 * k + 1] = wy;
      w.U[3 * k + 2] = wz;
      Us[3 * k] = wx;
      Us[3 * k + 1] = wy;
      Us[3 * k + 2] = wz;
    }
    double cs[3] = {cx.part(), cy.part(), cz.part()};
    cta_sum<3>(cs, sh, par);  // also completes Xs and Us for the objective
    const double inv_n = ty.inv_n;
    const V3<S> cvol{(S)(cs[0] * inv_n), (S)(cs[1] * inv_n), (S)(cs[2] * inv_n)};
    NPFEM_PHASE_END(t_predict, kPhPredict, P, tid)
    NPFEM_PHASE_BEGIN(t_obj0)
    const CtaEval ev = cta_objective<S, kLim ? 1 : 0>(ty, P, w, Xs, Us, Gs, w.G, nullptr, cvol, cell, sh, par);
    NPFEM_PHASE_END(t_obj0, kPhObjective, P, tid)
    if (tid == 0) {
      st->fx = ev.energy;
      st->g0n = sqrt(ev.gg);
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
    if (iters == 0) {
      cta_finalize<S>(ty, P, st, Xs, Us, ev.gg, cell, 0, x, v);
      continue;
    }
    if (tid == 0) P.act_out[atomicAdd(P.act_count_out, 1)] = item;
    // the history is empty here, so the first half of the two-loop recursion is Q = g
    NPFEM_PHASE_BEGIN(t_loop1)
    for (int e = tid; e < len; e += nt) w.Q[e] = Gs[e];
    NPFEM_PHASE_END(t_loop1, kPhTwoLoop, P, tid)
  }
}

// One quasi-Newton iteration of every cell of the list still iterating, one cell per CTA
// at a time, after k_solve left r = A^-1 q in Q: second half of the two-loop recursion
// (fused with the first line-search trial), backtracking line search on the shared-memory
// objective, history update, then the first half of the next iteration's recursion or
// the write-back.
template <typename S, bool kLim>
__global__ void __launch_bounds__(32 * kIterCtaMaxWarps, IterCtaOccupancy<S>::min_blocks)
    npfem_k_iter_cta(DevTypeView<S> ty, StepParams P, S* x, S* v) {
  extern __shared__ __align__(16) unsigned char cta_smem[];
  __shared__ CtaShared sh;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n = ty.n, len = 3 * n;
  S* Xs = reinterpret_cast<S*>(cta_smem);
  S* Us = Xs + len;
  S* Gs = Us + len;
  int par = 0;
  for (;;) {
    if (tid == 0) sh.item = atomicAdd(P.queue_counter, 1);
    __syncthreads();
    const int item = sh.item;
    __syncthreads();
    if (item >= P.ncells_list) break;
    const int cell = P.cell_list[item];
    char* base = P.scratch + (size_t)item * P.slot_bytes;
    CellState<S>* st = reinterpret_cast<CellState<S>*>(base);
    const int k = st->k, iters = st->iters;
    if (k >= iters) continue;  // same header for the whole CTA: a uniform branch
    CellWs<S> w = split_ws<S>(base, ty);
    const int cur = st->cur;
    const S* U = cur ? w.UT : w.U;
    S* UT = cur ? w.U : w.UT;
    const S* G = cur ? w.GT : w.G;
    S* GT = cur ? w.G : w.GT;
    const V3<S> cvol{st->cvol[0], st->cvol[1], st->cvol[2]};
    const double fx = st->fx;
    int hcount = st->hcount, hhead = st->hhead;
    for (int e = tid; e < len; e += nt) Xs[e] = w.X[e];
    NPFEM_PHASE_BEGIN(t_loop2)
    // Second half, oldest -> newest pairs: each pass applies one pair's update and
    // accumulates the next pair's y . Q; the last pass writes D = -Q with g . D and the
    // line search's first trial U + D.
    double gd;
    {
      Acc<S> agd;
      if (hcount == 0) {
        for (int e = tid; e < len; e += nt) {
          const S d = -w.Q[e];
          w.D[e] = d;
          agd.add_prod(G[e], d);
          const S ut = U[e] + d;
          UT[e] = ut;
          Us[e] = ut;
        }
      } else {
        // r = A^-1 q from the solve is staged in the shared Gs (free until the line search)
        // by the first pass, and the passes update it there
        // pair k (oldest first) is slot (hhead - hcount + k) mod m; the pass of pair k reads
        // s_k and y_{k+1} (the last pass s_k, g and U), and fetches the next pass's vectors
        auto slot = [&](int k) { return (hhead - hcount + k + kHistory) % kHistory; };
        auto prefetch_pass = [&](int k) {
          if (k >= hcount) return;
          prefetch_l2(w.hs + (size_t)slot(k) * len, len, tid, nt);
          if (k + 1 < hcount) {
            prefetch_l2(w.hy + (size_t)slot(k + 1) * len, len, tid, nt);
          } else {
            prefetch_l2(G, len, tid, nt);
            prefetch_l2(U, len, tid, nt);
          }
        };
        int i = slot(0);
        S acc = 0;
        prefetch_pass(0);
        {
          const S* yi = w.hy + (size_t)i * len;
          for (int e = tid; e < len; e += nt) {
            const S qe = w.Q[e];
            Gs[e] = qe;
            acc += yi[e] * qe;
          }
        }
        for (int q = hcount - 1; q >= 0; --q) {
          const int k = hcount - 1 - q;
          prefetch_pass(k + 1);
          const S b = st->rho[i] * cta_sum_s<S>(acc, sh, par);
          const S c = st->aco[i] - b;
          const S* si = w.hs + (size_t)i * len;
          if (q > 0) {
            const int inext = (hhead - 1 - (q - 1) + kHistory) % kHistory;
            acc = update_dot<S>(Gs, c, si, w.hy + (size_t)inext * len, len, tid, nt);
            i = inext;
          } else {
            cta_negate_trial<S>(Gs, c, si, G, U, w.D, UT, Us, agd, len, tid, nt);
          }
        }
      }
      gd = cta_sum1(agd.part(), sh, par);
    }
    NPFEM_PHASE_END(t_loop2, kPhTwoLoop, P, tid)
    if (!(gd < 0.0)) {  // not a descent direction: drop history, plain PD step (rare)
      hcount = 0;
      hhead = 0;
      if (tid < 32) global_solve<S>(ty, w.z, false, G, w.Q, tid, false);
      __syncthreads();
      Acc<S> a2;
      for (int e = tid; e < len; e += nt) {
        const S d = -w.Q[e];
        w.D[e] = d;
        a2.add_prod(G[e], d);
        const S ut = U[e] + d;
        UT[e] = ut;
        Us[e] = ut;
      }
      gd = cta_sum1(a2.part(), sh, par);
    }
    double alpha = 1.0, ft = 0.0, gg = 0.0;
    bool degen = false;
    int status = 0;
    for (int h = 0; h <= kMaxHalvings; ++h) {
      if (h > 0) {
        const S sa = (S)alpha;
        for (int e = tid; e < len; e += nt) {
          const S ut = U[e] + sa * w.D[e];
          UT[e] = ut;
          Us[e] = ut;
        }
      }
      __syncthreads();
      NPFEM_PHASE_BEGIN(t_obj)
      const CtaEval et = cta_objective<S, kLim ? 1 : 0>(ty, P, w, Xs, Us, Gs, GT, w.D, cvol, cell, sh, par);
      NPFEM_PHASE_END(t_obj, kPhObjective, P, tid)
      ft = et.energy;
      gg = et.gg;
      degen = et.degenerate;  // the trial that ends the search is the accepted one
      const bool armijo = ft <= fx + kArmijoC1 * alpha * gd;
      const bool approx = (et.gtd <= (2.0 * kArmijoC1 - 1.0) * gd) && (ft <= fx + kEnergyGuardEps * fabs(fx));
      if (armijo || approx) break;
      if (h == kMaxHalvings) {
        status |= 1;
        break;
      }
      alpha *= 0.5;
    }
    // converged-residual mode: the accepted trial ends the step when |g| < tol |g0|
    const bool stop = P.tol > 0.0 && sqrt(gg) < P.tol * st->g0n;
    NPFEM_PHASE_BEGIN(t_hist)
    S new_rho = (S)0;
    bool keep = false;
    S sg = 0;  // this thread's part of s . g, the first dot of the next first half if the pair is kept
    if (k < iters - 1 && !stop) {
      // the accepted trial is in Us and Gs: s = UT - U, y = GT - G
      S* si = w.hs + (size_t)hhead * len;
      S* yi = w.hy + (size_t)hhead * len;
      Acc<S> asy, ass, ayy;
      for (int e = tid; e < len; e += nt) {
        const S g = Gs[e];
        const S s = Us[e] - U[e];
        const S y = g - G[e];
        si[e] = s;
        yi[e] = y;
        asy.add_prod(s, y);
        ass.add_prod(s, s);
        ayy.add_prod(y, y);
        sg += s * g;
      }
      double r3[3] = {asy.part(), ass.part(), ayy.part()};
      cta_sum<3>(r3, sh, par);
      // the curvature test and 1 / (s . y): scalar FP64 work, by thread 0 alone (the
      // barrier below publishes the decision)
      if (tid == 0 && r3[0] > kCurvatureEps * sqrt(r3[1]) * sqrt(r3[2])) {
        keep = true;
        new_rho = (S)(1.0 / r3[0]);
      }
    }
    NPFEM_PHASE_END(t_hist, kPhHistory, P, tid)
    if (P.alpha_log && k < P.alpha_log_len && tid == 0) P.alpha_log[(size_t)cell * P.alpha_log_len + k] = alpha;
    const int slot = hhead;
    if (tid == 0) {
      sh.keep = keep;
      const int hh = keep ? (hhead + 1) % kHistory : hhead;
      const int hc = keep ? (hcount < kHistory ? hcount + 1 : kHistory) : hcount;
      if (keep) st->rho[slot] = new_rho;
      st->hcount = hc;
      st->hhead = hh;
      st->fx = ft;
      st->cur = cur ^ 1;
      st->k = k + 1;
      st->status |= status;
      if (degen) st->degen = 1;
    }
    __syncthreads();  // the header (rho of the new pair) and the decision before the first half reads them
    keep = sh.keep != 0;
    if (keep) {
      hhead = (hhead + 1) % kHistory;
      hcount = hcount < kHistory ? hcount + 1 : kHistory;
    }
    // the accepted trial (UT, GT) is the new current iterate
    if (k + 1 < iters && !stop) {
      if (tid == 0) P.act_out[atomicAdd(P.act_count_out, 1)] = item;
      NPFEM_PHASE_BEGIN(t_loop1)
      cta_two_loop_first<S>(w, st, hcount, hhead, Gs, len, sh, par, keep ? &sg : nullptr);
      NPFEM_PHASE_END(t_loop1, kPhTwoLoop, P, tid)
    } else {
      cta_finalize<S>(ty, P, st, Xs, Us, gg, cell, k + 1, x, v);
    }
  }
}

}  // namespace npfem
