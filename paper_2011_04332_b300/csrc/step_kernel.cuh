// Device code of the npFEM batched step: one warp advances one cell by one time step.
//
// Per cell (npFEM solid step, Implementation and architecture section of the paper;
// quasi-Newton projective dynamics of Liu et al. 2017 named there):
//   K1  y = x_n + dt v_n + dt^2 M^-1 f_ext, x^(0) = y           (prediction, Eq. (2))
//   K2  f(x) and grad f(x): per-triangle strain projections, per-hinge bending
//       projections, global area/volume terms, inertia; gradient gathered per vertex
//   K3  L-BFGS two-loop recursion, history 5
//   K4  H0 = A^-1 by the per-type FP64 LDL^T factor: permute, unit-lower forward
//       solve, diagonal scaling, unit-upper backward solve (3 right-hand sides)
//   K5  backtracking line search (K2 at every trial point)
//   K6  history update and FP64 residual / energy reductions
//   K7  v_{n+1} = (x_{n+1} - x_n)/dt, write back
//
// Everything a warp needs for its cell lives in its workspace slot (global memory,
// L1/L2 resident) except the FP64 solve vector, which sits in shared memory when it
// fits.  All intra-cell synchronisation is warp-level (__syncwarp, shuffles).
// Positions are handled as x = anchor + X + U where anchor is the cell's first input
// vertex, X = x_n - anchor and U is the displacement of the step, so that FP32 work
// never subtracts two large nearby coordinates.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "npfem_internal.h"

namespace npfem {

constexpr unsigned kFull = 0xffffffffu;

struct StepParams {
  int ncells_list;             // cells handled by this launch
  const int32_t* cell_list;    // [ncells_list] cell ids (batch order)
  const int64_t* offsets;      // [ncells+1] vertex offsets
  int64_t n_total;
  const int32_t* iters;        // [ncells] or null
  int iters_default;
  double* residual_out;        // [ncells] or null
  int32_t* status_out;         // [ncells] or null
  double tol;                  // > 0: stop a cell once |g| < tol |g0| (converged-residual mode)
  int32_t* iters_done;         // [ncells] iterations run, or null
  const int32_t* contact_count;  // [N_total] contact planes per vertex (0..2), or null: no collisions
  const double* contact_plane;   // [N_total][2][4] unit normal, offset relative to the cell's anchor
  double contact_delta, contact_weight;  // penalty (w/2) max(0, delta - gap)^2 per plane
  const double* box;           // with collisions and walls: [6] box lo, hi (absolute); else null
  const void* x_state;         // the state being stepped (S*): each cell's anchor is its first vertex
  double* alpha_log;           // [ncells][alpha_log_len] or null
  int alpha_log_len;
  int* queue_counter;          // work-queue head (zeroed before the launch)
  char* scratch;               // workspace, slot_bytes per warp
  size_t slot_bytes;
  int z_in_smem;               // 1: FP64 solve vector in dynamic shared memory
  int solve_per_coord;         // 1: sweep x, y, z one after another with a one-coordinate vector
  int solve_cells;             // split mode: cells a warp of the solve kernel sweeps together (1..4)
  const int* act_in;           // split mode: list of cells iterating at this iteration (one-warp k_solve)
  const int* act_count_in;     //   and its length
  int* act_out;                // split mode: list of cells iterating at the next iteration
  int* act_count_out;          //   (appended by k_begin / k_iter) and its length
  unsigned long long* phase_cycles;  // [kPhases] per-phase SM cycles summed over warps
};

// Per-phase cycle telemetry (when the batch counts phases, P.phase_cycles non-null): each
// warp (CTA) adds the SM clock cycles it spent in a phase to a batch-owned counter (one
// relaxed 64-bit atomic by lane (thread) 0 per phase instance).
enum Phase { kPhPredict = 0, kPhObjective, kPhTwoLoop, kPhSolve, kPhHistory, kPhWrite, kPhAreaVolume, kPhGather,
             kPhases = 8 };
#define NPFEM_PHASE_BEGIN(var) const long long var = clock64();
#define NPFEM_PHASE_END(var, ph, P, lane) \
  if ((lane) == 0 && (P).phase_cycles) atomicAdd(&(P).phase_cycles[ph], (unsigned long long)(clock64() - (var)));

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
template <typename S>
__device__ __forceinline__ S warp_sum(S v);
template <>
__device__ __forceinline__ float warp_sum<float>(float v) { return warp_sum_f(v); }
template <>
__device__ __forceinline__ double warp_sum<double>(double v) { return warp_sum_d(v); }

// Per-lane accumulator for sums that are reduced in FP64 across the warp.  For FP32
// terms it keeps an unevaluated (hi, lo) pair updated with error-free transformations
// (TwoSum; TwoProd through fmaf), so a lane's partial sum carries ~48 significant bits
// on the FP32 pipe; the lane totals are then combined in FP64.  For FP64 terms it is a
// plain double.
template <typename S>
struct Acc;
template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double part() const { return s; }
  __device__ __forceinline__ double total() const { return warp_sum_d(s); }
};
template <>
struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    float t = hi + x;
    float bb = t - hi;
    lo += (hi - (t - bb)) + (x - bb);
    hi = t;
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    float p = a * b;
    float e = fmaf(a, b, -p);
    add(p);
    lo += e;
  }
  __device__ __forceinline__ double part() const { return (double)hi + (double)lo; }  // this lane's sum
  __device__ __forceinline__ double total() const { return warp_sum_d(part()); }
};

template <typename S>
struct V3 {
  S x, y, z;
};
template <typename S>
__device__ __forceinline__ V3<S> ld3(const S* p, int i) {
  return {p[3 * i], p[3 * i + 1], p[3 * i + 2]};
}
template <typename S>
__device__ __forceinline__ void st3(S* p, int i, V3<S> v) {
  p[3 * i] = v.x;
  p[3 * i + 1] = v.y;
  p[3 * i + 2] = v.z;
}
// Four consecutive entries of a per-element table with 4 entries per element (16-byte
// aligned rows: one vector load for floats and ints, two for doubles).
struct Q4f {
  float x, y, z, w;
};
struct Q4d {
  double x, y, z, w;
};
template <typename S>
struct Q4Of;
template <>
struct Q4Of<float> {
  using type = Q4f;
};
template <>
struct Q4Of<double> {
  using type = Q4d;
};
__device__ __forceinline__ Q4f ldg4(const float* p) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  return {a.x, a.y, a.z, a.w};
}
__device__ __forceinline__ Q4d ldg4(const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ int4 ldg4(const int32_t* p) { return __ldg(reinterpret_cast<const int4*>(p)); }

template <typename S>
__device__ __forceinline__ V3<S> operator+(V3<S> a, V3<S> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <typename S>
__device__ __forceinline__ V3<S> operator-(V3<S> a, V3<S> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename S>
__device__ __forceinline__ V3<S> operator*(S s, V3<S> a) { return {s * a.x, s * a.y, s * a.z}; }
template <typename S>
__device__ __forceinline__ V3<S> cross(V3<S> a, V3<S> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <typename S>
__device__ __forceinline__ S dot(V3<S> a, V3<S> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Edge vector x_b - x_a from the rest-relative start positions X and displacement U.
template <typename S>
__device__ __forceinline__ V3<S> edge(const S* X, const S* U, int a, int b) {
  return (ld3(X, b) - ld3(X, a)) + (ld3(U, b) - ld3(U, a));
}

// Per-cell workspace pointers (all arrays [n][3] of S unless noted).
template <typename S>
struct CellWs {
  S *X, *W, *U, *UT, *G, *GT, *D, *Q;
  S *hs, *hy;      // [m][3n]
  S *corner;       // [T][3][3] per-corner gradient of the triangle terms
  S *hbuf;         // [E][3] w_e (K - p)
  double* z;       // [n+1][3] FP64 solve vector (row n = padding sink)
};

template <typename S>
__device__ __forceinline__ size_t slot_bytes_for(int n, int T, int E, bool z_in_smem) {
  size_t v = (size_t)3 * n;
  size_t bytes = sizeof(S) * ((8 + 2 * kHistory) * v + 9 * (size_t)T + 3 * (size_t)E);
  bytes = (bytes + 255) & ~(size_t)255;
  if (!z_in_smem) bytes += sizeof(double) * 3 * ((size_t)n + 1);
  return (bytes + 255) & ~(size_t)255;
}

template <typename S>
__device__ __forceinline__ CellWs<S> carve(char* base, int n, int T, int E, double* zsmem) {
  CellWs<S> w;
  size_t v = (size_t)3 * n;
  S* p = reinterpret_cast<S*>(base);
  w.X = p; p += v;
  w.W = p; p += v;
  w.U = p; p += v;
  w.UT = p; p += v;
  w.G = p; p += v;
  w.GT = p; p += v;
  w.D = p; p += v;
  w.Q = p; p += v;
  w.hs = p; p += kHistory * v;
  w.hy = p; p += kHistory * v;
  w.corner = p; p += 9 * (size_t)T;
  w.hbuf = p; p += 3 * (size_t)E;
  if (zsmem) {
    w.z = zsmem;
  } else {
    size_t off = reinterpret_cast<char*>(p) - base;
    off = (off + 255) & ~(size_t)255;
    w.z = reinterpret_cast<double*>(base + off);
  }
  return w;
}

// ------------------------------------------------------------------ K2
// Incidence entries of a vertex loaded together by the gradient gather (pass D).
constexpr int kGatherBatch = 6;

struct EvalOut {
  double energy;
  bool degenerate;
};

// Box walls (cell-wall contact): each face of the box [lo, hi] acts on every vertex of the
// current iterate with (w/2) max(0, delta - gap)^2, gap the distance inside the box along
// the face's axis; positions relative to the cell's anchor (the first vertex of the stepped
// state, as in the step).  Adds to the gradient; returns the lane's share of the energy.
template <typename S>
__device__ __noinline__ double wall_pass(const S* xs, int64_t off, int64_t Nt, double dl, double wc,
                                         const double* box, const S* X, const S* U, S* G, int n, int lane,
                                         int stride = 32) {
  double lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    const double a = (double)xs[d * Nt + off];
    lo[d] = box[d] - a;
    hi[d] = box[3 + d] - a;
  }
  double e = 0.0;
  for (int v = lane; v < n; v += stride) {
    const V3<S> p = ld3(X, v) + ld3(U, v);
    const double q[3] = {(double)p.x, (double)p.y, (double)p.z};
    double f[3] = {0.0, 0.0, 0.0};
    bool any = false;
    for (int d = 0; d < 3; ++d) {
      const double pl = dl - (q[d] - lo[d]);
      if (pl > 0.0) {
        e += 0.5 * wc * pl * pl;
        f[d] -= wc * pl;
        any = true;
      }
      const double ph = dl - (hi[d] - q[d]);
      if (ph > 0.0) {
        e += 0.5 * wc * ph * ph;
        f[d] += wc * ph;
        any = true;
      }
    }
    if (any) {
      V3<S> g = ld3(G, v);
      g.x += (S)f[0];
      g.y += (S)f[1];
      g.z += (S)f[2];
      st3(G, v, g);
    }
  }
  return e;
}

// Rayleigh damping terms of the objective, out of line so that the iteration kernels'
// register allocation does not carry them when damping is off.  Each returns its lane's
// share of the damping energy.  Elastic part: per triangle (c_beta/dt) w_t |G_t U|^2 / 2
// with its corner gradients, per hinge (c_beta/dt) w_e |sum_j c_j U_j|^2 / 2 into the
// hinge buffer (the gather applies the c_j).
template <typename S>
__device__ __noinline__ double damping_elastic(const int32_t* tris, const S* Dinv, const S* w_tri,
                                               const int32_t* hinges, const S* c_hinge, const S* w_hinge, int T,
                                               int E, S dl, const S* U, S* corner, S* hbuf, int lane) {
  const S half = (S)0.5;
  double e = 0.0;
  for (int t = lane; t < T; t += 32) {
    const int i0 = __ldg(&tris[3 * t]), i1 = __ldg(&tris[3 * t + 1]), i2 = __ldg(&tris[3 * t + 2]);
    const V3<S> u0 = ld3(U, i0);
    const V3<S> u1 = ld3(U, i1) - u0, u2 = ld3(U, i2) - u0;
    const S d00 = __ldg(&Dinv[3 * t]), d01 = __ldg(&Dinv[3 * t + 1]), d11 = __ldg(&Dinv[3 * t + 2]);
    const S wd = dl * __ldg(&w_tri[t]);
    const V3<S> F0 = d00 * u1, F1 = d01 * u1 + d11 * u2;
    e += (double)(half * wd * (dot(F0, F0) + dot(F1, F1)));
    const V3<S> P0 = wd * F0, P1 = wd * F1;
    const V3<S> g1 = d00 * P0 + d01 * P1, g2 = d11 * P1;
    st3(corner, 3 * t + 0, ld3(corner, 3 * t + 0) - (g1 + g2));
    st3(corner, 3 * t + 1, ld3(corner, 3 * t + 1) + g1);
    st3(corner, 3 * t + 2, ld3(corner, 3 * t + 2) + g2);
  }
  for (int h = lane; h < E; h += 32) {
    const int i = __ldg(&hinges[4 * h]), j = __ldg(&hinges[4 * h + 1]);
    const int ka = __ldg(&hinges[4 * h + 2]), kb = __ldg(&hinges[4 * h + 3]);
    const S c1 = __ldg(&c_hinge[4 * h + 1]), c2 = __ldg(&c_hinge[4 * h + 2]), c3 = __ldg(&c_hinge[4 * h + 3]);
    const V3<S> ui = ld3(U, i);
    const V3<S> KU = c1 * (ld3(U, j) - ui) + c2 * (ld3(U, ka) - ui) + c3 * (ld3(U, kb) - ui);
    const S wd = dl * __ldg(&w_hinge[h]);
    e += (double)(half * wd * dot(KU, KU));
    st3(hbuf, h, ld3(hbuf, h) + wd * KU);
  }
  return e;
}

// Mass part: (c_alpha/dt) m_v |U_v|^2 / 2 per vertex, its gradient added to G.
template <typename S>
__device__ __noinline__ double damping_mass(const S* mass, int n, S dm, const S* U, S* G, int lane,
                                            int stride = 32) {
  double e = 0.0;
  for (int v = lane; v < n; v += stride) {
    const V3<S> u = ld3(U, v);
    const S md = dm * __ldg(&mass[v]);
    e += 0.5 * (double)md * (double)dot(u, u);
    st3(G, v, ld3(G, v) + md * u);
  }
  return e;
}

// Strain limits: projection of F = [F0 F1] (3x2) onto the matrices whose singular values
// lie in [s_min, s_max], R = F M with M = k2 I + (k1 - k2)/(l1 - l2) (C - l2 I), where
// l1 >= l2 are the eigenvalues of C = F^T F and k_i = clamp(sqrt(l_i))/sqrt(l_i) (the
// spectral projector of the 2x2 C in closed form; l1 - l2 = 2 disc exactly, equal
// eigenvalues give k1 = k2 and M = k2 I).  M is evaluated in FP64 in both forms, per
// triangle in a pass of its own that stores (m00, m01, m11) in the first three slots of
// the triangle's corner record; the strain pass, run by the same lane over the same
// triangles, reads them before it overwrites the record.  The pass runs at the top of the
// objective, where few values are live, so that types without limits keep the register
// allocation of the polar projection (a call inside the objective, or the FP64 projector
// inside the strain loop, would raise the spills of the iteration kernel).
template <typename S>
__device__ __forceinline__ void strain_limit_pass(const DevTypeView<S>& ty, const S* X, const S* U, S* corner,
                                               int lane, int stride = 32) {
  const double s_min = ty.s_min, s_max = ty.s_max;
  // margin of the inside test below, far above the rounding of its working precision
  const S lo2 = (S)(s_min * s_min * (1.0 + (sizeof(S) == 4 ? 1e-4 : 1e-12)));
  const S hi2 = (S)(s_max * s_max * (1.0 - (sizeof(S) == 4 ? 1e-4 : 1e-12)));
  for (int t = lane; t < ty.T; t += stride) {
    int i0 = __ldg(&ty.tris[3 * t]), i1 = __ldg(&ty.tris[3 * t + 1]), i2 = __ldg(&ty.tris[3 * t + 2]);
    V3<S> e1 = edge(X, U, i0, i1), e2 = edge(X, U, i0, i2);
    const S d00 = __ldg(&ty.Dinv[3 * t]), d01 = __ldg(&ty.Dinv[3 * t + 1]), d11 = __ldg(&ty.Dinv[3 * t + 2]);
    V3<S> F0 = d00 * e1;
    V3<S> F1 = d01 * e1 + d11 * e2;
    {
      // Both squared singular values clearly inside [s_min^2, s_max^2]: the clamp changes
      // nothing, k1 = k2 = 1 and the projector below yields M = I exactly, so it is skipped.
      // The test runs in the working precision (for the FP32 form an FP32 test instead of
      // an FP64 eigen-decomposition per triangle); near a limit, or for a degenerate F
      // (NaN or infinite quotient), the FP64 projector decides.
      const S c00s = dot(F0, F0), c01s = dot(F0, F1), c11s = dot(F1, F1);
      const S hs = (S)0.5 * (c00s + c11s), qs = (S)0.5 * (c00s - c11s);
      const S l1s = hs + sqrt(qs * qs + c01s * c01s);
      const V3<S> xs = cross(F0, F1);
      const S l2s = dot(xs, xs) / l1s;
      if (l2s > lo2 && l1s < hi2) {
        corner[9 * t] = (S)1;
        corner[9 * t + 1] = (S)0;
        corner[9 * t + 2] = (S)1;
        continue;
      }
    }
    const double a0 = F0.x, a1 = F0.y, a2 = F0.z, b0 = F1.x, b1 = F1.y, b2 = F1.z;
    const double c00 = a0 * a0 + a1 * a1 + a2 * a2;
    const double c01 = a0 * b0 + a1 * b1 + a2 * b2;
    const double c11 = b0 * b0 + b1 * b1 + b2 * b2;
    const double h = 0.5 * (c00 + c11), q = 0.5 * (c00 - c11);
    const double disc = sqrt(q * q + c01 * c01);
    // smaller eigenvalue as det C / l1, det C = |F0 x F1|^2 (Lagrange identity): h - disc
    // and c00 c11 - c01^2 both cancel for thin triangles; l2 = 0 (collinear F) gives M = I
    const double x0 = a1 * b2 - a2 * b1, x1 = a2 * b0 - a0 * b2, x2 = a0 * b1 - a1 * b0;
    const double l1 = h + disc, l2 = (x0 * x0 + x1 * x1 + x2 * x2) / l1;
    const bool ok = l2 > 0.0;
    const double s1 = sqrt(l1), s2 = ok ? sqrt(l2) : 1.0;
    const double k1 = ok ? fmin(fmax(s1, s_min), s_max) / s1 : 1.0;
    const double k2 = ok ? fmin(fmax(s2, s_min), s_max) / s2 : 1.0;
    const double coef = disc > 0.0 ? (k1 - k2) / (2.0 * disc) : 0.0;
    corner[9 * t] = (S)(k2 + coef * (c00 - l2));
    corner[9 * t + 1] = (S)(coef * c01);
    corner[9 * t + 2] = (S)(k2 + coef * (c11 - l2));
  }
}

// Strain, area and volume terms of one triangle: e1, e2 its edges from corner 0, q0 corner 0
// relative to the volume centre cvol, tc = (d00, d01, d11, w_t), kA and kV the area and
// volume penalty slopes.  Adds the strain energy w_t/2 |F - R|^2 to e_el, sets degen for a
// degenerate F^T F, and returns the gradients at the three corners.  mrec: the triangle's
// strain-limit matrix (m00, m01, m11), R = F M, for a limited type; null: R = F (F^T F)^-1/2
// by the closed-form 2x2 SPD square root (C + sqrt(det C) I)/sqrt(tr C + 2 sqrt(det C)).
template <typename S>
__device__ __forceinline__ void triangle_terms(V3<S> e1, V3<S> e2, V3<S> q0, const typename Q4Of<S>::type& tc,
                                               const S* mrec, S kA, S kV, Acc<S>& e_el, bool& degen, V3<S>& g0,
                                               V3<S>& g1, V3<S>& g2) {
  const S half = (S)0.5, sixth = (S)(1.0 / 6.0);
  const S d00 = tc.x, d01 = tc.y, d11 = tc.z;
  const S wt = tc.w;
  V3<S> F0 = d00 * e1;
  V3<S> F1 = d01 * e1 + d11 * e2;
  S c00 = dot(F0, F0), c01 = dot(F0, F1), c11 = dot(F1, F1);
  S det = c00 * c11 - c01 * c01;
  V3<S> P0{0, 0, 0}, P1{0, 0, 0};
  // the threshold in the element's own precision: an FP64 compare per element would load
  // the FP32 form's FP64 pipe, which the solves need (1e-30 is a normal FP32 number)
  if (det > (S)kDegenerateDet) {
    V3<S> R0, R1;
    if (mrec) {
      const S m00 = mrec[0], m01 = mrec[1], m11 = mrec[2];
      R0 = m00 * F0 + m01 * F1;
      R1 = m01 * F0 + m11 * F1;
    } else {
      S s = sqrt(det);
      S tau = sqrt(c00 + c11 + (S)2 * s);
      S s00 = (c00 + s) / tau, s01 = c01 / tau, s11 = (c11 + s) / tau;
      S idet = (S)1 / (s00 * s11 - s01 * s01);
      // R = F S^-1, S^-1 = [[s11, -s01], [-s01, s00]] / det S
      R0 = idet * (s11 * F0 - s01 * F1);
      R1 = idet * (s00 * F1 - s01 * F0);
    }
    V3<S> D0 = F0 - R0, D1 = F1 - R1;
    e_el.add(half * wt * (dot(D0, D0) + dot(D1, D1)));
    P0 = wt * D0;
    P1 = wt * D1;
  } else {
    degen = true;
  }
  // strain: dE/de1 = P0 d00 + P1 d01, dE/de2 = P1 d11
  g1 = d00 * P0 + d01 * P1;
  g2 = d11 * P1;
  g0 = (S)-1 * (g1 + g2);
  // area: dA_t/dx_k = n/2 x (x_{k+2} - x_{k+1})
  V3<S> N = cross(e1, e2);
  S nn = sqrt(dot(N, N));
  if (nn > (S)0) {
    V3<S> nh = ((S)1 / nn) * N;
    g0 = g0 + (kA * half) * cross(nh, e2 - e1);
    g1 = g1 + (kA * half) * cross(nh, (S)-1 * e2);
    g2 = g2 + (kA * half) * cross(nh, e1);
  }
  // volume: dV_t/dq0 = q1 x q2 / 6 (cyclic), q = x - cvol
  V3<S> q1 = q0 + e1, q2 = q0 + e2;
  g0 = g0 + (kV * sixth) * cross(q1, q2);
  g1 = g1 + (kV * sixth) * cross(q2, q0);
  g2 = g2 + (kV * sixth) * cross(q0, q1);
}

// Hinge vector K = sum_j c_j x_j = c1 (x_j - x_i) + c2 (x_kA - x_i) + c3 (x_kB - x_i) of the
// hinge (i, j, kA, kB) with coefficients cv = (c0, c1, c2, c3).
template <typename S>
__device__ __forceinline__ V3<S> hinge_vector(const S* X, const S* U, int4 hv,
                                              const typename Q4Of<S>::type& cv) {
  return cv.y * edge(X, U, hv.x, hv.y) + cv.z * edge(X, U, hv.x, hv.z) + cv.w * edge(X, U, hv.x, hv.w);
}

// Bending term of one hinge: the projection p of K onto |K| = |K0| (K0row = (K0x, K0y,
// K0z, |K0|); p = K0 when |K| vanishes), w_e/2 |K - p|^2 added to e_el.  Returns w_e (K - p),
// whose product with c_j is the gradient at the hinge's vertex j.
template <typename S>
__device__ __forceinline__ V3<S> hinge_terms(V3<S> K, const S* K0row, S we, Acc<S>& e_el) {
  S kn = sqrt(dot(K, K));
  V3<S> p;
  if (kn < (S)kDegenerateNorm) {
    p = {__ldg(&K0row[0]), __ldg(&K0row[1]), __ldg(&K0row[2])};
  } else {
    p = (__ldg(&K0row[3]) / kn) * K;
  }
  V3<S> r = K - p;
  e_el.add((S)0.5 * we * dot(r, r));
  return we * r;
}

// f(X+U) and its gradient into Gout.  W = y - x_n.  The strain projection maps the
// triangle deformation gradient F = [e1 e2] Dm^-1 to R = F (F^T F)^(-1/2) via the
// closed-form 2x2 SPD square root (C + sqrt(det C) I)/sqrt(tr C + 2 sqrt(det C)).
// kLim: 0 compiles the rotations only, 1 the strain-limited projection only, 2 chooses by
// the type at run time (the split kernels are instantiated per case, so a batch without
// limits runs code with no trace of them).
template <typename S, int kLim = 2>
__device__ EvalOut eval_objective(const DevTypeView<S>& ty, const StepParams& P, const CellWs<S>& w, const S* U,
                                  S* Gout, V3<S> cvol, int cell, int lane) {
  const int n = ty.n, T = ty.T, E = ty.E;
  const S* X = w.X;
  const bool limited = kLim == 1 || (kLim == 2 && ty.limited);
  if (limited) strain_limit_pass<S>(ty, X, U, w.corner, lane);
  NPFEM_PHASE_BEGIN(t_area)
  // pass A: global area and volume (FP64 reductions)
  Acc<S> a_sum, v_sum;
  for (int t = lane; t < T; t += 32) {
    const int4 tv = ldg4(ty.tri4 + 4 * t);
    const int i0 = tv.x, i1 = tv.y, i2 = tv.z;
    V3<S> e1 = edge(X, U, i0, i1), e2 = edge(X, U, i0, i2);
    V3<S> N = cross(e1, e2);
    a_sum.add(sqrt(dot(N, N)));
    V3<S> q0 = (ld3(X, i0) + ld3(U, i0)) - cvol;
    v_sum.add(dot(q0, N));
  }
  const double A = 0.5 * a_sum.total();
  const double V = v_sum.total() / 6.0;
  const double dA = A - ty.A0, dV = V - ty.V0;
  const double e_area = 0.5 * ty.w_area * dA * dA / ty.A0;
  const double e_vol = 0.5 * ty.w_vol * dV * dV / ty.V0;
  const S kA = (S)(ty.w_area * dA / ty.A0);
  const S kV = (S)(ty.w_vol * dV / ty.V0);
  const S half = (S)0.5;

  NPFEM_PHASE_END(t_area, kPhAreaVolume, P, lane)
  // pass B: triangles (strain projection + area/volume corner gradients)
  Acc<S> e_el;
  bool degen = false;
  for (int t = lane; t < T; t += 32) {
    const int4 tv = ldg4(ty.tri4 + 4 * t);
    const typename Q4Of<S>::type tc = ldg4(ty.trc + 4 * t);
    const int i0 = tv.x, i1 = tv.y, i2 = tv.z;
    const V3<S> e1 = edge(X, U, i0, i1), e2 = edge(X, U, i0, i2);
    const V3<S> q0 = (ld3(X, i0) + ld3(U, i0)) - cvol;
    V3<S> g0, g1, g2;
    triangle_terms<S>(e1, e2, q0, tc, limited ? w.corner + 9 * t : nullptr, kA, kV, e_el, degen, g0, g1, g2);
    st3(w.corner, 3 * t + 0, g0);
    st3(w.corner, 3 * t + 1, g1);
    st3(w.corner, 3 * t + 2, g2);
  }

  // pass C: hinges (bending projection onto |K| = |K0|)
  for (int h = lane; h < E; h += 32) {
    const int4 hv = ldg4(ty.hinges + 4 * h);
    const typename Q4Of<S>::type cv = ldg4(ty.c_hinge + 4 * h);
    const V3<S> K = hinge_vector<S>(X, U, hv, cv);
    st3(w.hbuf, h, hinge_terms<S>(K, ty.K0 + 4 * h, __ldg(&ty.w_hinge[h]), e_el));
  }
  // Rayleigh damping, elastic part: (c_beta/dt)/2 U^T L U with U = x - x_n, element by
  // element into the same corner and hinge buffers (each owned by the lane that wrote it)
  if (ty.damp_l != 0.0)
    e_el.add((S)damping_elastic<S>(ty.tris, ty.Dinv, ty.w_tri, ty.hinges, ty.c_hinge, ty.w_hinge, T, E,
                                   (S)ty.damp_l, U, w.corner, w.hbuf, lane));
  __syncwarp();

  NPFEM_PHASE_BEGIN(t_gather)
  // pass D: vertices (inertia + gather of element contributions)
  const S idt2 = (S)(1.0 / (ty.dt * ty.dt));
  for (int v = lane; v < n; v += 32) {
    V3<S> du = ld3(U, v) - ld3(w.W, v);
    const S m = __ldg(&ty.mass[v]);
    e_el.add(half * m * idt2 * dot(du, du));
    V3<S> g = (m * idt2) * du;
    const int e0 = __ldg(&ty.inc_ptr[v]), e1 = __ldg(&ty.inc_ptr[v + 1]);
    // The vertex's entries (its corners, then its hinge entries) kGatherBatch at a time:
    // every code of a batch, then every record it names, is loaded before the first add,
    // so a lane has a batch of independent loads in flight instead of one round trip per
    // entry.  The adds keep the entry order; a corner adds 1 * record, which rounds like
    // the plain add.  Records are addressed from the corner array, which the hinge
    // buffer follows (hbuf = corner + 9T).
    for (int e = e0; e < e1; e += kGatherBatch) {
      int off[kGatherBatch];
      S cf[kGatherBatch];
#pragma unroll
      for (int k = 0; k < kGatherBatch; ++k) {
        const int ek = e + k < e1 ? e + k : e1 - 1;
        const int code = __ldg(&ty.inc_code[ek]);
        off[k] = code >= 0 ? 3 * code : 9 * T + 3 * ((-code - 1) >> 2);
        cf[k] = code >= 0 ? (S)1 : __ldg(&ty.inc_coef[ek]);
      }
      V3<S> rec[kGatherBatch];
#pragma unroll
      for (int k = 0; k < kGatherBatch; ++k) rec[k] = {w.corner[off[k]], w.corner[off[k] + 1], w.corner[off[k] + 2]};
#pragma unroll
      for (int k = 0; k < kGatherBatch; ++k)
        if (e + k < e1) g = g + cf[k] * rec[k];
    }
    st3(Gout, v, g);
  }
  // Rayleigh damping, mass part: (c_alpha/dt)/2 sum_v m_v |U_v|^2 (same vertex per lane)
  if (ty.damp_m != 0.0) e_el.add((S)damping_mass<S>(ty.mass, n, (S)ty.damp_m, U, Gout, lane));
  NPFEM_PHASE_END(t_gather, kPhGather, P, lane)
  EvalOut o;
  o.energy = e_el.total() + e_area + e_vol;
  if (P.contact_count) {
    // pass E: contact planes (fixed for the step), (w/2) max(0, delta - gap)^2 each, on
    // the vertices that have any; a pass of its own keeps pass D's registers unchanged
    __syncwarp();
    const int64_t off = P.offsets[cell];
    double e_ct = 0.0;
    for (int v = lane; v < n; v += 32) {
      const int nc = P.contact_count[off + v];
      if (nc == 0) continue;
      V3<S> g = ld3(Gout, v);
      const V3<S> p = ld3(X, v) + ld3(U, v);
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
      st3(Gout, v, g);
    }
    o.energy += warp_sum_d(e_ct);
    // box walls (cell-wall contact), out of line: a step without walls carries none of it
    if (P.box)
      o.energy += warp_sum_d(wall_pass<S>(static_cast<const S*>(P.x_state), off, P.n_total, P.contact_delta,
                                          P.contact_weight, P.box, X, U, Gout, n, lane));
  }
  o.degenerate = __any_sync(kFull, degen);
  __syncwarp();
  return o;
}

// ------------------------------------------------------------------ vector helpers
template <typename S>
__device__ __forceinline__ S vdot(const S* a, const S* b, int len, int lane) {
  S s = 0;
  for (int i = lane; i < len; i += 32) s += a[i] * b[i];
  return warp_sum<S>(s);
}
template <typename S>
__device__ __forceinline__ double vdot64(const S* a, const S* b, int len, int lane) {
  Acc<S> s;
  for (int i = lane; i < len; i += 32) s.add_prod(a[i], b[i]);
  return s.total();
}

// ------------------------------------------------------------------ K4
// One triangular sweep: chunks of 32 updates z[row] -= val * z[col], one per lane,
// packed on the host so that every source is final before its chunk and targets are
// distinct; the warp synchronises only before chunks flagged as hazardous.  The chunk
// tables stream from L2 and are prefetched kPrefetch chunks ahead in registers.  When
// the solve vector is in shared memory it is addressed through the shared window.
constexpr int kPrefetch = 8;

__device__ __forceinline__ double lds_f64(uint32_t a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts_f64(uint32_t a, double v) {
  asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

// One triangular sweep (Eqs. (7)-(8): the prefactored global step) over the packed
// 32-entry chunks of L, applied to kCells solve vectors at once: cells of one type
// share L, so every entry (r, j, l) loaded from the factor stream updates
// z_c[r] -= l * z_c[j] for all kCells cells and kComp coordinates.  Each z_c is its
// own array ([n+1][kComp]: row n is the pad row of inactive lanes), so every shared
// memory access keeps the bank pattern the chunk packing was scheduled for.
template <bool kShared, int kComp, int kCells>
__device__ __forceinline__ void chunk_sweep_n(int nc, const int32_t* __restrict__ meta,
                                              const uint32_t* __restrict__ rc, const double* __restrict__ val,
                                              double* const* z, int n, int lane) {
  uint32_t zs[kCells];
#pragma unroll
  for (int c = 0; c < kCells; ++c) zs[c] = kShared ? (uint32_t)__cvta_generic_to_shared(z[c]) : 0u;
  int mb[kPrefetch];
  uint32_t eb[kPrefetch];
  double vb[kPrefetch];
#pragma unroll
  for (int k = 0; k < kPrefetch; ++k) {
    if (k < nc) {
      mb[k] = __ldg(meta + k);
      eb[k] = __ldg(rc + (size_t)k * kChunk + lane);
      vb[k] = __ldg(val + (size_t)k * kChunk + lane);
    } else {
      mb[k] = 0;
      eb[k] = (uint32_t)n | ((uint32_t)n << 16);
      vb[k] = 0.0;
    }
  }
  for (int base = 0; base < nc; base += kPrefetch) {
#pragma unroll
    for (int k = 0; k < kPrefetch; ++k) {
      const int ch = base + k;
      if (ch < nc) {
        const int m = mb[k];
        const uint32_t e = eb[k];
        const double l = vb[k];
        const int nx = ch + kPrefetch;
        if (nx < nc) {
          mb[k] = __ldg(meta + nx);
          eb[k] = __ldg(rc + (size_t)nx * kChunk + lane);
          vb[k] = __ldg(val + (size_t)nx * kChunk + lane);
        }
        if (m & 1) __syncwarp();
        const int r = (int)(e & 0xffffu), j = (int)(e >> 16);
        double xj[kCells][kComp], zr[kCells][kComp];
        if (kShared) {
          const uint32_t oj = 8u * kComp * (uint32_t)j, orr = 8u * kComp * (uint32_t)r;
#pragma unroll
          for (int c = 0; c < kCells; ++c)
#pragma unroll
            for (int d = 0; d < kComp; ++d) xj[c][d] = lds_f64(zs[c] + oj + 8 * d);
#pragma unroll
          for (int c = 0; c < kCells; ++c)
#pragma unroll
            for (int d = 0; d < kComp; ++d) zr[c][d] = fma(-l, xj[c][d], lds_f64(zs[c] + orr + 8 * d));
#pragma unroll
          for (int c = 0; c < kCells; ++c)
#pragma unroll
            for (int d = 0; d < kComp; ++d) sts_f64(zs[c] + orr + 8 * d, zr[c][d]);
        } else {
#pragma unroll
          for (int c = 0; c < kCells; ++c)
#pragma unroll
            for (int d = 0; d < kComp; ++d) xj[c][d] = z[c][kComp * j + d];
#pragma unroll
          for (int c = 0; c < kCells; ++c)
#pragma unroll
            for (int d = 0; d < kComp; ++d) zr[c][d] = fma(-l, xj[c][d], z[c][kComp * r + d]);
#pragma unroll
          for (int c = 0; c < kCells; ++c)
#pragma unroll
            for (int d = 0; d < kComp; ++d) z[c][kComp * r + d] = zr[c][d];
        }
      }
    }
  }
  __syncwarp();
}

// R = A^-1 Q for kCells cells of one type and kComp coordinates per vector: permute,
// unit-lower forward sweep, D^-1 scaling, unit-upper backward sweep, all in FP64.
template <bool kShared, int kComp, int kCells, bool kBlocked, typename View>
__device__ void solve_components_n(const View& ty, double* const* z, int n, int lane) {
  chunk_sweep_n<kShared, kComp, kCells>(ty.nchunks_fwd, ty.fwd_meta, ty.fwd_rc, ty.fwd_val, z, n, lane);
  constexpr int B = kBlocked ? 4 : 1;
#pragma unroll 1
  for (int r0 = 0; r0 < n; r0 += 32 * B) {
    double d[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int r = r0 + 32 * u + lane;
      d[u] = r < n ? __ldg(&ty.dinv[r]) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int r = r0 + 32 * u + lane;
      if (r < n)
#pragma unroll
        for (int c = 0; c < kCells; ++c)
#pragma unroll
          for (int q = 0; q < kComp; ++q) z[c][kComp * r + q] *= d[u];
    }
  }
  __syncwarp();
  chunk_sweep_n<kShared, kComp, kCells>(ty.nchunks_bwd, ty.bwd_meta, ty.bwd_rc, ty.bwd_val, z, n, lane);
}

// Rows per lane per block of the permuted gather / scatter and of the D^-1 scaling
// (kBlocked): every load of a block is issued before any of its stores, so a lane has
// several independent global loads in flight instead of one round trip per row (the
// compiler cannot move the loads past stores to possibly aliasing vectors).  The price
// is registers, so only the solve kernel of the split mode takes it.
template <int kCells, bool kBlocked>
struct GatherBlock {
  static constexpr int value = !kBlocked ? 1 : (kCells >= 3 ? 1 : (kCells == 2 ? 2 : 4));
};

// z[c][kComp r + q] = Q[c][3 perm[r] + q0 + q] for the rows of the type (q0 = 0 and
// kComp = 3, or one coordinate q0 with kComp = 1); pad row n = 0.
template <typename S, int kCells, int kComp, bool kBlocked>
__device__ __forceinline__ void gather_rhs(const DevTypeView<S>& ty, double* const* z, const S* const* Q, int q0,
                                           int lane) {
  constexpr int B = GatherBlock<kCells, kBlocked>::value;
  const int n = ty.n;
#pragma unroll 1
  for (int r0 = 0; r0 < n; r0 += 32 * B) {
    int v[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int r = r0 + 32 * u + lane;
      v[u] = r < n ? __ldg(&ty.perm[r]) : -1;
    }
    S q[B][kCells][kComp];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (v[u] >= 0)
#pragma unroll
        for (int c = 0; c < kCells; ++c)
#pragma unroll
          for (int d = 0; d < kComp; ++d) q[u][c][d] = Q[c][3 * v[u] + q0 + d];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (v[u] >= 0) {
        const int r = r0 + 32 * u + lane;
#pragma unroll
        for (int c = 0; c < kCells; ++c)
#pragma unroll
          for (int d = 0; d < kComp; ++d) z[c][kComp * r + d] = (double)q[u][c][d];
      }
  }
  if (lane < kComp)
#pragma unroll
    for (int c = 0; c < kCells; ++c) z[c][kComp * n + lane] = 0.0;
}

// R[c][3 perm[r] + q0 + q] = z[c][kComp r + q], rounded to S.
template <typename S, int kCells, int kComp, bool kBlocked>
__device__ __forceinline__ void scatter_result(const DevTypeView<S>& ty, double* const* z, S* const* R, int q0,
                                               int lane) {
  constexpr int B = GatherBlock<kCells, kBlocked>::value;
  const int n = ty.n;
#pragma unroll 1
  for (int r0 = 0; r0 < n; r0 += 32 * B) {
    int v[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
      const int r = r0 + 32 * u + lane;
      v[u] = r < n ? __ldg(&ty.perm[r]) : -1;
    }
    S o[B][kCells][kComp];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (v[u] >= 0) {
        const int r = r0 + 32 * u + lane;
#pragma unroll
        for (int c = 0; c < kCells; ++c)
#pragma unroll
          for (int d = 0; d < kComp; ++d) o[u][c][d] = (S)z[c][kComp * r + d];
      }
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (v[u] >= 0)
#pragma unroll
        for (int c = 0; c < kCells; ++c)
#pragma unroll
          for (int d = 0; d < kComp; ++d) R[c][3 * v[u] + q0 + d] = o[u][c][d];
  }
}

// Global solve of kCells cells of one type (Q[c] -> R[c] = A^-1 Q[c], Q and R may
// alias), the three coordinates interleaved in z[c] ([n+1][3]) or, per_coord with the
// vectors in shared memory, swept one after another through one-coordinate vectors
// ([n+1]); both orders do the same FP64 operations per coordinate.
template <typename S, int kCells, bool kBlocked = false>
__device__ void global_solve_n(const DevTypeView<S>& ty, double* const* z, bool z_shared, const S* const* Q,
                               S* const* R, int lane, bool per_coord) {
  const int n = ty.n;
  if (!per_coord || !z_shared) {
    gather_rhs<S, kCells, 3, kBlocked>(ty, z, Q, 0, lane);
    __syncwarp();
    if (z_shared)
      solve_components_n<true, 3, kCells, kBlocked>(ty, z, n, lane);
    else
      solve_components_n<false, 3, kCells, kBlocked>(ty, z, n, lane);
    scatter_result<S, kCells, 3, kBlocked>(ty, z, R, 0, lane);
    __syncwarp();
    return;
  }
  for (int q = 0; q < 3; ++q) {
    gather_rhs<S, kCells, 1, kBlocked>(ty, z, Q, q, lane);
    __syncwarp();
    solve_components_n<true, 1, kCells, kBlocked>(ty, z, n, lane);
    scatter_result<S, kCells, 1, kBlocked>(ty, z, R, q, lane);
    __syncwarp();
  }
}

template <typename S>
__device__ void global_solve(const DevTypeView<S>& ty, double* z, bool z_shared, const S* Q, S* R, int lane,
                             bool per_coord = false) {
  double* zz[1] = {z};
  const S* qq[1] = {Q};
  S* rr[1] = {R};
  global_solve_n<S, 1>(ty, zz, z_shared, qq, rr, lane, per_coord);
}

// ------------------------------------------------------------------ one cell
// Forward record kept for the adjoint (tape mode): iterates and gradients of every
// accepted quasi-Newton iteration, step lengths, and per-iteration flags.
struct TapeRec {
  double* U;      // [maxk+1][3n] displacement iterates U_k (x_k = x_n + U_k)
  double* G;      // [maxk+1][3n] gradients g_k
  double* alpha;  // [maxk] accepted step lengths
  int* flags;     // [maxk] bit 0: history cleared before the direction; bit 1: pair (s_k, y_k) kept
};
constexpr int kTapeReset = 1, kTapeKept = 2;

template <typename S>
__device__ __forceinline__ void copy_vec(S* dst, const S* src, int len, int lane) {
  for (int i = lane; i < len; i += 32) dst[i] = src[i];
}

// One cell, one step.  kTape = true (FP64 only) records the forward pass into `tape`
// for the adjoint and writes no output state.
template <typename S, bool kTape = false>
__device__ void process_cell(const DevTypeView<S>& ty, const StepParams& P, const CellWs<S>& w, int cell,
                             S* x, S* v, const S* f, int lane, const TapeRec* tape = nullptr) {
  const int n = ty.n;
  const int len = 3 * n;
  const int64_t off = P.offsets[cell];
  const int64_t Nt = P.n_total;
  const int iters = P.iters ? P.iters[cell] : P.iters_default;
  const double dt = ty.dt;
  const S sdt = (S)dt, sdt2 = (S)(dt * dt);

  NPFEM_PHASE_BEGIN(t_predict)
  // K1: anchor, X = x_n - anchor, W = y - x_n, U = W
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

  S* U = w.U;
  S* UT = w.UT;
  S* G = w.G;
  S* GT = w.GT;
  NPFEM_PHASE_END(t_predict, kPhPredict, P, lane)
  NPFEM_PHASE_BEGIN(t_obj0)
  EvalOut ev = eval_objective<S>(ty, P, w, U, G, cvol, cell, lane);
  NPFEM_PHASE_END(t_obj0, kPhObjective, P, lane)
  double fx = ev.energy;
  bool degen = false;  // set by accepted iterates only
  if (kTape) {
    copy_vec<double>(tape->U, (const double*)U, len, lane);
    copy_vec<double>(tape->G, (const double*)G, len, lane);
  }
  const double g0n = sqrt(vdot64<S>(G, G, len, lane));
  int status = 0;
  int hcount = 0, hhead = 0;
  S rho[kHistory], aco[kHistory];
#pragma unroll
  for (int i = 0; i < kHistory; ++i) rho[i] = aco[i] = 0;

  int done = iters;
  for (int k = 0; k < iters; ++k) {
    NPFEM_PHASE_BEGIN(t_loop1)
    // K3 first loop: Q = G; newest -> oldest
    for (int i = lane; i < len; i += 32) w.Q[i] = G[i];
    __syncwarp();
    for (int q = 0; q < hcount; ++q) {
      int i = (hhead - 1 - q + kHistory) % kHistory;
      const S* si = w.hs + (size_t)i * len;
      const S* yi = w.hy + (size_t)i * len;
      S a = rho[i] * vdot<S>(si, w.Q, len, lane);
      aco[i] = a;
      for (int e = lane; e < len; e += 32) w.Q[e] -= a * yi[e];
      __syncwarp();
    }
    // K4: r = H0 q
    NPFEM_PHASE_END(t_loop1, kPhTwoLoop, P, lane)
    NPFEM_PHASE_BEGIN(t_solve)
    global_solve<S>(ty, w.z, P.z_in_smem != 0, w.Q, w.Q, lane, P.solve_per_coord != 0);
    NPFEM_PHASE_END(t_solve, kPhSolve, P, lane)
    NPFEM_PHASE_BEGIN(t_loop2)
    // K3 second loop: oldest -> newest
    for (int q = hcount - 1; q >= 0; --q) {
      int i = (hhead - 1 - q + kHistory) % kHistory;
      const S* si = w.hs + (size_t)i * len;
      const S* yi = w.hy + (size_t)i * len;
      S b = rho[i] * vdot<S>(yi, w.Q, len, lane);
      S c = aco[i] - b;
      for (int e = lane; e < len; e += 32) w.Q[e] += c * si[e];
      __syncwarp();
    }
    for (int e = lane; e < len; e += 32) w.D[e] = -w.Q[e];
    __syncwarp();
    double gd = vdot64<S>(G, w.D, len, lane);
    NPFEM_PHASE_END(t_loop2, kPhTwoLoop, P, lane)
    if (kTape && lane == 0) tape->flags[k] = 0;
    if (!(gd < 0.0)) {  // not a descent direction: drop history, plain PD step
      hcount = 0;
      hhead = 0;
      if (kTape && lane == 0) tape->flags[k] |= kTapeReset;
      global_solve<S>(ty, w.z, P.z_in_smem != 0, G, w.Q, lane, P.solve_per_coord != 0);
      for (int e = lane; e < len; e += 32) w.D[e] = -w.Q[e];
      __syncwarp();
      gd = vdot64<S>(G, w.D, len, lane);
    }
    // K5: backtracking line search
    double alpha = 1.0, ft = 0.0;
    bool trial_degen = false;
    for (int h = 0; h <= kMaxHalvings; ++h) {
      const S sa = (S)alpha;
      for (int e = lane; e < len; e += 32) UT[e] = U[e] + sa * w.D[e];
      __syncwarp();
      NPFEM_PHASE_BEGIN(t_obj)
      EvalOut et = eval_objective<S>(ty, P, w, UT, GT, cvol, cell, lane);
      NPFEM_PHASE_END(t_obj, kPhObjective, P, lane)
      ft = et.energy;
      trial_degen = et.degenerate;
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
    degen = degen || trial_degen;  // the trial that ends the search is the accepted one
    // converged-residual mode: the accepted trial ends the step when |g| < tol |g0|
    const bool stop = P.tol > 0.0 && sqrt(vdot64<S>(GT, GT, len, lane)) < P.tol * g0n;
    NPFEM_PHASE_BEGIN(t_hist)
    // K6: history pair (s, y) = (UT - U, GT - G) into the ring slot hhead
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
        if (kTape && lane == 0) tape->flags[k] |= kTapeKept;
        rho[hhead] = (S)(1.0 / sy);
        hhead = (hhead + 1) % kHistory;
        hcount = hcount < kHistory ? hcount + 1 : kHistory;
      }
      __syncwarp();
    }
    NPFEM_PHASE_END(t_hist, kPhHistory, P, lane)
    if (P.alpha_log && k < P.alpha_log_len && lane == 0) P.alpha_log[(size_t)cell * P.alpha_log_len + k] = alpha;
    // accept
    S* t1 = U;
    U = UT;
    UT = t1;
    S* t2 = G;
    G = GT;
    GT = t2;
    fx = ft;
    if (kTape) {
      copy_vec<double>(tape->U + (size_t)(k + 1) * len, (const double*)U, len, lane);
      copy_vec<double>(tape->G + (size_t)(k + 1) * len, (const double*)G, len, lane);
      if (lane == 0) tape->alpha[k] = alpha;
      __syncwarp();
    }
    if (stop) {
      done = k + 1;
      break;
    }
  }

  NPFEM_PHASE_BEGIN(t_write)
  if (kTape) {
    __syncwarp();
    return;
  }
  // K7: residual, write x_{n+1} = anchor + X + U and v_{n+1} = U / dt
  const double gn = sqrt(vdot64<S>(G, G, len, lane));
  const S idt = (S)(1.0 / dt);
  bool bad = false;
  for (int k = lane; k < n; k += 32) {
    double nx = (double)ax + ((double)w.X[3 * k] + (double)U[3 * k]);
    double ny = (double)ay + ((double)w.X[3 * k + 1] + (double)U[3 * k + 1]);
    double nz = (double)az + ((double)w.X[3 * k + 2] + (double)U[3 * k + 2]);
    S vx = U[3 * k] * idt, vy = U[3 * k + 1] * idt, vz = U[3 * k + 2] * idt;
    x[off + k] = (S)nx;
    x[Nt + off + k] = (S)ny;
    x[2 * Nt + off + k] = (S)nz;
    v[off + k] = vx;
    v[Nt + off + k] = vy;
    v[2 * Nt + off + k] = vz;
    bad = bad || !isfinite(nx) || !isfinite(ny) || !isfinite(nz) || !isfinite((double)vx) ||
          !isfinite((double)vy) || !isfinite((double)vz);
  }
  bad = __any_sync(kFull, bad);
  NPFEM_PHASE_END(t_write, kPhWrite, P, lane)
  if (lane == 0) {
    if (degen) status |= 2;
    if (bad) status |= 4;
    if (P.status_out) P.status_out[cell] = status;
    if (P.residual_out) P.residual_out[cell] = g0n > 0.0 ? gn / g0n : 0.0;
    if (P.iters_done) P.iters_done[cell] = done;
  }
  __syncwarp();
}

// Persistent kernel: each warp owns one workspace slot and pops cells from the queue.
template <typename S>
__global__ void __launch_bounds__(128) npfem_step_kernel(DevTypeView<S> ty, StepParams P, S* x, S* v,
                                                          const S* f) {
  extern __shared__ double smem_z[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int slot = blockIdx.x * (blockDim.x >> 5) + wib;
  const int zc = P.solve_per_coord ? 1 : 3;
  double* zs = P.z_in_smem ? smem_z + (size_t)wib * zc * (ty.n + 1) : nullptr;
  CellWs<S> w = carve<S>(P.scratch + (size_t)slot * P.slot_bytes, ty.n, ty.T, ty.E, zs);
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(P.queue_counter, 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= P.ncells_list) break;
    process_cell<S>(ty, P, w, P.cell_list[item], x, v, f, lane);
  }
}

}  // namespace npfem
