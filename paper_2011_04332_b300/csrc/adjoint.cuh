// Reverse mode of one npFEM step (K8), FP64: a CTA per cell for the unrolled iteration,
// a warp per cell for the implicit-function adjoint.
//
// The forward step is the quasi-Newton projective-dynamics iteration of the paper's
// solid solver (Liu et al. 2017, named in the Implementation and architecture
// section) run for a fixed number of iterations.  Its derivative is taken through the
// unrolled iteration with the accepted line-search step lengths held fixed (they are
// piecewise constant in the inputs):
//   y = x_n + dt v_n + dt^2 M^-1 f,  x_0 = y,  g_k = grad f(x_k; y, w),
//   d_k = -H_k g_k (two-loop recursion over the kept pairs, H0 = A(w)^-1),
//   x_{k+1} = x_k + alpha_k d_k,  s_k = x_{k+1} - x_k,  y_k = g_{k+1} - g_k,
//   x_{n+1} = x_K,  v_{n+1} = (x_K - x_n)/dt.
// Inputs: dL/dx_{n+1}, dL/dv_{n+1}.  Outputs: dL/dx_n, dL/dv_n, dL/df and dL/dw for the
// four material weights (strain, bending, area, volume).  The forward pass is recomputed
// with a tape (process_cell<double, true>); the reverse sweep needs Hessian-vector
// products of f, including the derivative of the polar projection R = F (F^T F)^-1/2:
// with S = (F^T F)^1/2, dR = dF S^-1 - R dS S^-1 where S dS + dS S = dC solves in
// closed form for 2x2 SPD S as dS = (dC + det(S) S^-1 dC S^-1) / (2 tr(S)).
#pragma once
#include "iter_cta.cuh"
#include "step_kernel.cuh"

namespace npfem {

constexpr int kMaxAdjIters = 16;

struct AdjParams {
  const double* gx_next;  // [3][Nt] dL/dx_{n+1}
  const double* gv_next;  // [3][Nt] dL/dv_{n+1} (may be null)
  double* gx;             // [3][Nt] out dL/dx_n
  double* gv;             // [3][Nt] out dL/dv_n
  double* gf;             // [3][Nt] out dL/df
  double* gw;             // [ncells][4] out dL/d(w_strain, w_bend, w_area, w_vol)
  char* scratch;          // adjoint workspace, slot_bytes per warp
  size_t slot_bytes;
  double w_mat[4];        // material weights of this launch's type
};

// Per-warp adjoint workspace (all [3n] FP64 vectors unless noted).
struct AdjWs {
  TapeRec tape;
  double *gbar;      // [maxk+1][3n] dL/dg_k
  double *sP, *yP;   // [maxk][3n] pairs s_k, y_k
  double *sbar, *ybar;  // [maxk][3n]
  double *Qs, *Rs;   // [kHistory+1][3n] two-loop intermediates
  double *XB, *DB, *QB, *RB, *HV, *YB;
  double *rho, *rhobar;  // [maxk]
};

__device__ __forceinline__ size_t adj_slot_bytes(int n) {
  size_t v = (size_t)3 * n;
  size_t nvec = 3 * (size_t)(kMaxAdjIters + 1) + 4 * (size_t)kMaxAdjIters + 2 * (size_t)(kHistory + 1) + 6;
  return ((sizeof(double) * (nvec * v + 3 * kMaxAdjIters) + sizeof(int) * kMaxAdjIters) + 255) & ~(size_t)255;
}

__device__ __forceinline__ AdjWs carve_adj(char* base, int n) {
  AdjWs a;
  size_t v = (size_t)3 * n;
  double* p = reinterpret_cast<double*>(base);
  a.tape.U = p; p += (kMaxAdjIters + 1) * v;
  a.tape.G = p; p += (kMaxAdjIters + 1) * v;
  a.gbar = p; p += (kMaxAdjIters + 1) * v;
  a.sP = p; p += kMaxAdjIters * v;
  a.yP = p; p += kMaxAdjIters * v;
  a.sbar = p; p += kMaxAdjIters * v;
  a.ybar = p; p += kMaxAdjIters * v;
  a.Qs = p; p += (kHistory + 1) * v;
  a.Rs = p; p += (kHistory + 1) * v;
  a.XB = p; p += v;
  a.DB = p; p += v;
  a.QB = p; p += v;
  a.RB = p; p += v;
  a.HV = p; p += v;
  a.YB = p; p += v;
  a.tape.alpha = p; p += kMaxAdjIters;
  a.rho = p; p += kMaxAdjIters;
  a.rhobar = p; p += kMaxAdjIters;
  a.tape.flags = reinterpret_cast<int*>(p);
  return a;
}

__device__ __forceinline__ void vaxpy(double* y, double a, const double* x, int len, int lane) {
  for (int i = lane; i < len; i += 32) y[i] = fma(a, x[i], y[i]);
}
__device__ __forceinline__ void vzero(double* y, int len, int lane) {
  for (int i = lane; i < len; i += 32) y[i] = 0.0;
}

// The threads that work on one cell: a warp (the implicit adjoint) or a CTA (the unrolled
// adjoint's reverse sweep).  Element loops stride by size() from rank(); sync() orders the
// team's memory accesses; sums<K>() turn per-thread FP64 partials into totals every member
// receives (all members make the same sequence of calls); leader() writes per-cell
// scalars; solver() marks the warp that runs the warp-level FP64 solve (lane() its lane).
struct WarpTeam {
  int lane_;
  __device__ int rank() const { return lane_; }
  __device__ int size() const { return 32; }
  __device__ int lane() const { return lane_; }
  __device__ bool leader() const { return lane_ == 0; }
  __device__ bool solver() const { return true; }
  __device__ void sync() const { __syncwarp(); }
  template <int K>
  __device__ void sums(double (&v)[K]) const {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = warp_sum_d(v[k]);
  }
};
struct CtaTeam {
  CtaShared* sh;
  int* par;
  __device__ int rank() const { return threadIdx.x; }
  __device__ int size() const { return blockDim.x; }
  __device__ int lane() const { return threadIdx.x & 31; }
  __device__ bool leader() const { return threadIdx.x == 0; }
  __device__ bool solver() const { return threadIdx.x < 32; }
  __device__ void sync() const { __syncthreads(); }
  template <int K>
  __device__ void sums(double (&v)[K]) const {
    cta_sum<K>(v, *sh, *par);
  }
};

template <class Tm>
__device__ __forceinline__ double team_sum(const Tm& T, double x) {
  double v[1] = {x};
  T.sums(v);
  return v[0];
}
template <class Tm>
__device__ __forceinline__ void tvaxpy(const Tm& T, double* y, double a, const double* x, int len) {
  for (int i = T.rank(); i < len; i += T.size()) y[i] = fma(a, x[i], y[i]);
}
template <class Tm>
__device__ __forceinline__ void tvzero(const Tm& T, double* y, int len) {
  for (int i = T.rank(); i < len; i += T.size()) y[i] = 0.0;
}
// a . b: plain products (as vdot) or through the FP64 accumulator (as vdot64)
template <class Tm>
__device__ __forceinline__ double tdot(const Tm& T, const double* a, const double* b, int len) {
  double s = 0;
  for (int i = T.rank(); i < len; i += T.size()) s += a[i] * b[i];
  return team_sum(T, s);
}
template <class Tm>
__device__ __forceinline__ double tdot64(const Tm& T, const double* a, const double* b, int len) {
  Acc<double> s;
  for (int i = T.rank(); i < len; i += T.size()) s.add_prod(a[i], b[i]);
  return team_sum(T, s.part());
}
// The warp-level solve Q <- A^-1 Q run by the team's solver warp, visible to the team after.
template <class Tm>
__device__ __forceinline__ void team_solve(const Tm& T, const DevTypeView<double>& ty, const CellWs<double>& w,
                                           const StepParams& P, const double* in, double* out) {
  if (T.solver()) global_solve<double>(ty, w.z, P.z_in_smem != 0, in, out, T.lane(), P.solve_per_coord != 0);
  T.sync();
}

template <class Tm>
__device__ void matrix_weight_forms(const DevTypeView<double>& ty, const double* a, const double* b, double* fs,
                                    double* fb, const Tm& T);
template <class Tm>
__device__ void apply_rayleigh(const DevTypeView<double>& ty, const CellWs<double>& w, const double* a,
                               double* out, const Tm& T);

// Strain limits: the projection P = U clamp(Sigma, lo, hi) V^T of F = [F0 F1] and its
// directional derivative dP along dF, given the polar factor R = F (F^T F)^-1/2 and its
// derivative dR.  By regime of the two singular values: both inside the limits, P = F and
// dP = dF; both clamped to the same limit L, P = L R and dP = L dR (well conditioned for
// any eigenvalue gap); otherwise (one on each side, so the eigenvalues l1 > l2 of
// C = F^T F are apart) the spectral form P = F M, M = k2 I + c (C - l2 I),
// c = (k1 - k2)/(l1 - l2), k_i = clamp(s_i)/s_i, differentiated with
// dl1 = tr(Pi1 dC), Pi1 = (C - l2 I)/(l1 - l2), dl2 = tr(dC) - dl1, dk_i = -L/(2 s_i^3) dl_i
// for a clamped s_i (0 inside), dc = (dk1 - dk2)/(l1 - l2) - (k1 - k2)(dl1 - dl2)/(l1 - l2)^2,
// dM = dk2 I + dc (C - l2 I) + c (dC - dl2 I), dP = dF M + F dM.  Regimes and
// eigenvalues as in the step's limit pass (l2 = |F0 x F1|^2 / l1, l1 - l2 = 2 disc).
__device__ __noinline__ void limited_projection_jvp(V3<double> F0, V3<double> F1, V3<double> dF0, V3<double> dF1,
                                                    V3<double> R0, V3<double> R1, V3<double> dR0,
                                                    V3<double> dR1, double lo, double hi, V3<double>* P0,
                                                    V3<double>* P1, V3<double>* dP0, V3<double>* dP1) {
  const double c00 = dot(F0, F0), c01 = dot(F0, F1), c11 = dot(F1, F1);
  const double h = 0.5 * (c00 + c11), q = 0.5 * (c00 - c11);
  const double disc = sqrt(q * q + c01 * c01);
  const V3<double> fx = cross(F0, F1);
  const double l1 = h + disc, l2 = dot(fx, fx) / l1;
  const double s1 = sqrt(l1), s2 = sqrt(l2);
  const int r1 = s1 > hi ? 1 : (s1 < lo ? -1 : 0), r2 = s2 > hi ? 1 : (s2 < lo ? -1 : 0);
  if (r1 == 0 && r2 == 0) {
    *P0 = F0, *P1 = F1, *dP0 = dF0, *dP1 = dF1;
    return;
  }
  if (r1 == r2) {
    const double L = r1 > 0 ? hi : lo;
    *P0 = L * R0, *P1 = L * R1, *dP0 = L * dR0, *dP1 = L * dR1;
    return;
  }
  const double g00 = 2.0 * dot(F0, dF0), g01 = dot(F0, dF1) + dot(dF0, F1), g11 = 2.0 * dot(F1, dF1);
  const double gap = 2.0 * disc;
  const double dl1 = ((c00 - l2) * g00 + 2.0 * c01 * g01 + (c11 - l2) * g11) / gap;
  const double dl2 = g00 + g11 - dl1;
  const double L1 = r1 > 0 ? hi : lo, L2 = r2 > 0 ? hi : lo;
  const double k1 = r1 ? L1 / s1 : 1.0, k2 = r2 ? L2 / s2 : 1.0;
  const double dk1 = r1 ? -L1 / (2.0 * s1 * l1) * dl1 : 0.0, dk2 = r2 ? -L2 / (2.0 * s2 * l2) * dl2 : 0.0;
  const double c = (k1 - k2) / gap;
  const double dc = (dk1 - dk2) / gap - (k1 - k2) * (dl1 - dl2) / (gap * gap);
  const double m00 = k2 + c * (c00 - l2), m01 = c * c01, m11 = k2 + c * (c11 - l2);
  const double dm00 = dk2 + dc * (c00 - l2) + c * (g00 - dl2), dm01 = dc * c01 + c * g01,
               dm11 = dk2 + dc * (c11 - l2) + c * (g11 - dl2);
  *P0 = m00 * F0 + m01 * F1;
  *P1 = m01 * F0 + m11 * F1;
  *dP0 = (m00 * dF0 + m01 * dF1) + (dm00 * F0 + dm01 * F1);
  *dP1 = (m01 * dF0 + m11 * dF1) + (dm01 * F0 + dm11 * F1);
}

// Hessian-vector product out = grad^2 f(x) Vv at x = x_n + U (inertia and Rayleigh damping
// included), and wd[q] = Vv . d(grad f)/d(w_q) for the four material weights.  With strain
// limits the strain term differentiates the clamped projection (limited_projection_jvp).
template <class Tm>
__device__ void hessian_vector(const DevTypeView<double>& ty, const CellWs<double>& w, const double* U,
                               const double* Vv, double* out, V3<double> cvol, double wd[4], const Tm& Tm_) {
  const int n = ty.n, T = ty.T, E = ty.E;
  const double* X = w.X;
  Acc<double> a_sum, v_sum, da_sum, dv_sum, ws_sum, wb_sum;
  for (int t = Tm_.rank(); t < T; t += Tm_.size()) {
    int i0 = __ldg(&ty.tris[3 * t]), i1 = __ldg(&ty.tris[3 * t + 1]), i2 = __ldg(&ty.tris[3 * t + 2]);
    V3<double> e1 = edge(X, U, i0, i1), e2 = edge(X, U, i0, i2);
    V3<double> v0 = ld3(Vv, i0), de1 = ld3(Vv, i1) - v0, de2 = ld3(Vv, i2) - v0;
    V3<double> N = cross(e1, e2), dN = cross(de1, e2) + cross(e1, de2);
    double nn = sqrt(dot(N, N));
    a_sum.add(nn);
    if (nn > 0.0) da_sum.add(dot(N, dN) / nn);
    V3<double> q0 = (ld3(X, i0) + ld3(U, i0)) - cvol;
    v_sum.add(dot(q0, N));
    dv_sum.add(dot(v0, N) + dot(q0, dN));
  }
  double sv[4] = {a_sum.part(), v_sum.part(), da_sum.part(), dv_sum.part()};
  Tm_.sums(sv);
  const double A = 0.5 * sv[0], V = sv[1] / 6.0;
  const double dAv = 0.5 * sv[2], dVv = sv[3] / 6.0;
  const double kA = ty.w_area * (A - ty.A0) / ty.A0, kV = ty.w_vol * (V - ty.V0) / ty.V0;
  const double cA = ty.w_area / ty.A0 * dAv, cV = ty.w_vol / ty.V0 * dVv;
  wd[2] = (A - ty.A0) / ty.A0 * dAv;
  wd[3] = (V - ty.V0) / ty.V0 * dVv;

  for (int t = Tm_.rank(); t < T; t += Tm_.size()) {
    int i0 = __ldg(&ty.tris[3 * t]), i1 = __ldg(&ty.tris[3 * t + 1]), i2 = __ldg(&ty.tris[3 * t + 2]);
    V3<double> e1 = edge(X, U, i0, i1), e2 = edge(X, U, i0, i2);
    V3<double> vv0 = ld3(Vv, i0), vv1 = ld3(Vv, i1), vv2 = ld3(Vv, i2);
    V3<double> de1 = vv1 - vv0, de2 = vv2 - vv0;
    const double d00 = __ldg(&ty.Dinv[3 * t]), d01 = __ldg(&ty.Dinv[3 * t + 1]), d11 = __ldg(&ty.Dinv[3 * t + 2]);
    const double wt = __ldg(&ty.w_tri[t]), at = __ldg(&ty.tri_area[t]);
    V3<double> F0 = d00 * e1, F1 = d01 * e1 + d11 * e2;
    V3<double> dF0 = d00 * de1, dF1 = d01 * de1 + d11 * de2;
    double c00 = dot(F0, F0), c01 = dot(F0, F1), c11 = dot(F1, F1);
    double det = c00 * c11 - c01 * c01;
    V3<double> P0{0, 0, 0}, P1{0, 0, 0};
    if (det > kDegenerateDet) {
      double s = sqrt(det), tau = sqrt(c00 + c11 + 2.0 * s);
      double s00 = (c00 + s) / tau, s01 = c01 / tau, s11 = (c11 + s) / tau;
      double dS_ = s00 * s11 - s01 * s01, trS = s00 + s11;
      double i00 = s11 / dS_, i01 = -s01 / dS_, i11 = s00 / dS_;  // S^-1
      V3<double> R0 = i00 * F0 + i01 * F1, R1 = i01 * F0 + i11 * F1;
      // dC = dF^T F + F^T dF
      double g00 = 2.0 * dot(F0, dF0), g01 = dot(F0, dF1) + dot(dF0, F1), g11 = 2.0 * dot(F1, dF1);
      // M = S^-1 dC S^-1
      double t00 = i00 * g00 + i01 * g01, t01 = i00 * g01 + i01 * g11;
      double t10 = i01 * g00 + i11 * g01, t11 = i01 * g01 + i11 * g11;
      double m00 = t00 * i00 + t01 * i01, m01 = t00 * i01 + t01 * i11, m11 = t10 * i01 + t11 * i11;
      // dS = (dC + det(S) M) / (2 tr(S))
      const double i2t = 0.5 / trS;
      double h00 = (g00 + dS_ * m00) * i2t, h01 = (g01 + dS_ * m01) * i2t, h11 = (g11 + dS_ * m11) * i2t;
      // dR = dF S^-1 - R dS S^-1;  N = dS S^-1
      double n00 = h00 * i00 + h01 * i01, n01 = h00 * i01 + h01 * i11;
      double n10 = h01 * i00 + h11 * i01, n11 = h01 * i01 + h11 * i11;
      V3<double> dR0 = (i00 * dF0 + i01 * dF1) - (n00 * R0 + n10 * R1);
      V3<double> dR1 = (i01 * dF0 + i11 * dF1) - (n01 * R0 + n11 * R1);
      if (ty.limited)
        limited_projection_jvp(F0, F1, dF0, dF1, R0, R1, dR0, dR1, ty.s_min, ty.s_max, &R0, &R1, &dR0, &dR1);
      P0 = wt * (dF0 - dR0);
      P1 = wt * (dF1 - dR1);
      ws_sum.add(at * (dot(dF0, F0 - R0) + dot(dF1, F1 - R1)));
    }
    V3<double> g1 = d00 * P0 + d01 * P1;
    V3<double> g2 = d11 * P1;
    V3<double> g0 = -1.0 * (g1 + g2);
    // area: kA * d(grad A_t)[v] + cA * grad A_t
    V3<double> N = cross(e1, e2), dN = cross(de1, e2) + cross(e1, de2);
    double nn = sqrt(dot(N, N));
    if (nn > 0.0) {
      V3<double> nh = (1.0 / nn) * N;
      V3<double> dnh = (1.0 / nn) * (dN - dot(nh, dN) * nh);
      V3<double> a0 = cross(nh, e2 - e1), a1 = cross(nh, -1.0 * e2), a2 = cross(nh, e1);
      V3<double> b0 = cross(dnh, e2 - e1) + cross(nh, de2 - de1);
      V3<double> b1 = cross(dnh, -1.0 * e2) + cross(nh, -1.0 * de2);
      V3<double> b2 = cross(dnh, e1) + cross(nh, de1);
      g0 = g0 + (0.5 * kA) * b0 + (0.5 * cA) * a0;
      g1 = g1 + (0.5 * kA) * b1 + (0.5 * cA) * a1;
      g2 = g2 + (0.5 * kA) * b2 + (0.5 * cA) * a2;
    }
    // volume: kV * d(grad V_t)[v] + cV * grad V_t, q = x - cvol
    V3<double> q0 = (ld3(X, i0) + ld3(U, i0)) - cvol, q1 = q0 + e1, q2 = q0 + e2;
    const double sx = 1.0 / 6.0;
    g0 = g0 + (kV * sx) * (cross(vv1, q2) + cross(q1, vv2)) + (cV * sx) * cross(q1, q2);
    g1 = g1 + (kV * sx) * (cross(vv2, q0) + cross(q2, vv0)) + (cV * sx) * cross(q2, q0);
    g2 = g2 + (kV * sx) * (cross(vv0, q1) + cross(q0, vv1)) + (cV * sx) * cross(q0, q1);
    st3(w.corner, 3 * t + 0, g0);
    st3(w.corner, 3 * t + 1, g1);
    st3(w.corner, 3 * t + 2, g2);
  }
  for (int h = Tm_.rank(); h < E; h += Tm_.size()) {
    int i = __ldg(&ty.hinges[4 * h]), j = __ldg(&ty.hinges[4 * h + 1]);
    int ka = __ldg(&ty.hinges[4 * h + 2]), kb = __ldg(&ty.hinges[4 * h + 3]);
    const double c1 = __ldg(&ty.c_hinge[4 * h + 1]), c2 = __ldg(&ty.c_hinge[4 * h + 2]), c3 = __ldg(&ty.c_hinge[4 * h + 3]);
    V3<double> K = c1 * edge(X, U, i, j) + c2 * edge(X, U, i, ka) + c3 * edge(X, U, i, kb);
    V3<double> vi = ld3(Vv, i);
    V3<double> dK = c1 * (ld3(Vv, j) - vi) + c2 * (ld3(Vv, ka) - vi) + c3 * (ld3(Vv, kb) - vi);
    double kn = sqrt(dot(K, K));
    const double we = __ldg(&ty.w_hinge[h]), ue = __ldg(&ty.hinge_unit[h]);
    V3<double> hvec, p;
    if (kn < kDegenerateNorm) {
      p = {__ldg(&ty.K0[4 * h]), __ldg(&ty.K0[4 * h + 1]), __ldg(&ty.K0[4 * h + 2])};
      hvec = we * dK;
    } else {
      const double k0 = __ldg(&ty.K0[4 * h + 3]);
      V3<double> kh = (1.0 / kn) * K;
      p = k0 * kh;
      V3<double> dp = (k0 / kn) * (dK - dot(kh, dK) * kh);
      hvec = we * (dK - dp);
    }
    wb_sum.add(ue * dot(dK, K - p));
    st3(w.hbuf, h, hvec);
  }
  // Rayleigh damping: the quadratic (c_beta/dt) L and (c_alpha/dt) M terms, constant Hessians
  if (ty.damp_l != 0.0) {
    // the warp-level elastic damping terms, added to every element's record by the solver warp
    Tm_.sync();
    if (Tm_.solver())
      damping_elastic<double>(ty.tris, ty.Dinv, ty.w_tri, ty.hinges, ty.c_hinge, ty.w_hinge, T, E, ty.damp_l, Vv,
                              w.corner, w.hbuf, Tm_.lane());
  }
  Tm_.sync();
  const double idt2 = 1.0 / (ty.dt * ty.dt);
  for (int vtx = Tm_.rank(); vtx < n; vtx += Tm_.size()) {
    V3<double> g = (__ldg(&ty.mass[vtx]) * idt2) * ld3(Vv, vtx);
    const int e0 = __ldg(&ty.inc_ptr[vtx]), e1 = __ldg(&ty.inc_ptr[vtx + 1]);
    for (int e = e0; e < e1; ++e) {
      int code = __ldg(&ty.inc_code[e]);
      if (code >= 0)
        g = g + ld3(w.corner, code);
      else
        g = g + __ldg(&ty.inc_coef[e]) * ld3(w.hbuf, (-code - 1) >> 2);
    }
    st3(out, vtx, g);
  }
  if (ty.damp_m != 0.0) damping_mass<double>(ty.mass, n, ty.damp_m, Vv, out, Tm_.rank(), Tm_.size());
  double sw[2] = {ws_sum.part(), wb_sum.part()};
  Tm_.sums(sw);
  wd[0] = sw[0];
  wd[1] = sw[1];
  if (ty.damp_l != 0.0) {
    // d/dw of (c_beta/dt) L(w) U: the elastic matrix's weight forms between Vv and U
    double fs, fb;
    matrix_weight_forms(ty, Vv, U, &fs, &fb, Tm_);
    wd[0] += ty.damp_l * fs;
    wd[1] += ty.damp_l * fb;
  }
  Tm_.sync();
}

// Quadratic forms a^T (dA/dw_strain) b and a^T (dA/dw_bend) b of the global matrix.
template <class Tm>
__device__ void matrix_weight_forms(const DevTypeView<double>& ty, const double* a, const double* b, double* fs,
                                    double* fb, const Tm& Tm_) {
  Acc<double> ss, sb;
  for (int t = Tm_.rank(); t < ty.T; t += Tm_.size()) {
    int i0 = __ldg(&ty.tris[3 * t]), i1 = __ldg(&ty.tris[3 * t + 1]), i2 = __ldg(&ty.tris[3 * t + 2]);
    const double d00 = __ldg(&ty.Dinv[3 * t]), d01 = __ldg(&ty.Dinv[3 * t + 1]), d11 = __ldg(&ty.Dinv[3 * t + 2]);
    V3<double> a0 = ld3(a, i0), ae1 = ld3(a, i1) - a0, ae2 = ld3(a, i2) - a0;
    V3<double> b0 = ld3(b, i0), be1 = ld3(b, i1) - b0, be2 = ld3(b, i2) - b0;
    V3<double> aF0 = d00 * ae1, aF1 = d01 * ae1 + d11 * ae2;
    V3<double> bF0 = d00 * be1, bF1 = d01 * be1 + d11 * be2;
    ss.add(__ldg(&ty.tri_area[t]) * (dot(aF0, bF0) + dot(aF1, bF1)));
  }
  for (int h = Tm_.rank(); h < ty.E; h += Tm_.size()) {
    int i = __ldg(&ty.hinges[4 * h]), j = __ldg(&ty.hinges[4 * h + 1]);
    int ka = __ldg(&ty.hinges[4 * h + 2]), kb = __ldg(&ty.hinges[4 * h + 3]);
    const double c1 = __ldg(&ty.c_hinge[4 * h + 1]), c2 = __ldg(&ty.c_hinge[4 * h + 2]), c3 = __ldg(&ty.c_hinge[4 * h + 3]);
    V3<double> ai = ld3(a, i), bi = ld3(b, i);
    V3<double> Ka = c1 * (ld3(a, j) - ai) + c2 * (ld3(a, ka) - ai) + c3 * (ld3(a, kb) - ai);
    V3<double> Kb = c1 * (ld3(b, j) - bi) + c2 * (ld3(b, ka) - bi) + c3 * (ld3(b, kb) - bi);
    sb.add(__ldg(&ty.hinge_unit[h]) * dot(Ka, Kb));
  }
  double v[2] = {ss.part(), sb.part()};
  Tm_.sums(v);
  *fs = v[0];
  *fb = v[1];
}

// Reverse sweep of one cell after process_cell<double, true> filled the tape, by a team.
template <class Tm>
__device__ void reverse_cell(const DevTypeView<double>& ty, const StepParams& P, const AdjParams& A,
                             const CellWs<double>& w, const AdjWs& aw, int cell, int iters, const Tm& T) {
  const int n = ty.n, len = 3 * n;
  const int64_t off = P.offsets[cell], Nt = P.n_total;
  const double dt = ty.dt;
  const double* tU = aw.tape.U;
  const double* tG = aw.tape.G;
  Acc<double> cxa, cya, cza;
  for (int k = T.rank(); k < n; k += T.size()) {
    cxa.add(w.X[3 * k]);
    cya.add(w.X[3 * k + 1]);
    cza.add(w.X[3 * k + 2]);
  }
  double cs[3] = {cxa.part(), cya.part(), cza.part()};
  T.sums(cs);
  V3<double> cvol{cs[0] / n, cs[1] / n, cs[2] / n};
  double wacc[4] = {0, 0, 0, 0};
  const int K = iters;
  // pairs kept by the forward pass (identical arithmetic to the forward history update)
  for (int j = 0; j + 1 < K; ++j) {
    double* sj = aw.sP + (size_t)j * len;
    double* yj = aw.yP + (size_t)j * len;
    Acc<double> asy;
    for (int e = T.rank(); e < len; e += T.size()) {
      double s = tU[(size_t)(j + 1) * len + e] - tU[(size_t)j * len + e];
      double y = tG[(size_t)(j + 1) * len + e] - tG[(size_t)j * len + e];
      sj[e] = s;
      yj[e] = y;
      asy.add_prod(s, y);
    }
    double sy = team_sum(T, asy.part());
    if (T.leader()) aw.rho[j] = 1.0 / sy;
  }
  for (int k = 0; k <= K; ++k) tvzero(T, aw.gbar + (size_t)k * len, len);
  for (int j = 0; j < K; ++j) {
    tvzero(T, aw.sbar + (size_t)j * len, len);
    tvzero(T, aw.ybar + (size_t)j * len, len);
  }
  tvzero(T, aw.YB, len);
  // dL/dx_K = dL/dx_{n+1} + dL/dv_{n+1} / dt
  for (int k = T.rank(); k < n; k += T.size())
    for (int c = 0; c < 3; ++c) {
      double gxv = A.gx_next[c * Nt + off + k];
      double gvv = A.gv_next ? A.gv_next[c * Nt + off + k] : 0.0;
      aw.XB[3 * k + c] = gxv + gvv / dt;
    }
  T.sync();
  double wd[4];
  for (int k = K - 1; k >= 0; --k) {
    const int fl = aw.tape.flags[k];
    const double alpha = aw.tape.alpha[k];
    const double* xk1 = tU + (size_t)(k + 1) * len;
    double* gb1 = aw.gbar + (size_t)(k + 1) * len;
    double* gbk = aw.gbar + (size_t)k * len;
    // (1) pair k: s_k = x_{k+1} - x_k, y_k = g_{k+1} - g_k
    if (fl & kTapeKept) {
      const double* sb = aw.sbar + (size_t)k * len;
      const double* yb = aw.ybar + (size_t)k * len;
      for (int e = T.rank(); e < len; e += T.size()) {
        aw.XB[e] += sb[e];
        gb1[e] += yb[e];
        gbk[e] -= yb[e];
      }
      T.sync();
    }
    // (2) g_{k+1} = grad f(x_{k+1}): dL/dx_{k+1} += H gbar_{k+1}; dL/dy -= M/dt^2 gbar; weights
    hessian_vector(ty, w, xk1, gb1, aw.HV, cvol, wd, T);
    for (int q = 0; q < 4; ++q) wacc[q] += wd[q];
    for (int vtx = T.rank(); vtx < n; vtx += T.size()) {
      const double mi = __ldg(&ty.mass[vtx]) / (dt * dt);
      for (int c = 0; c < 3; ++c) {
        aw.XB[3 * vtx + c] += aw.HV[3 * vtx + c];
        aw.YB[3 * vtx + c] -= mi * gb1[3 * vtx + c];
      }
    }
    T.sync();
    // (3) x_{k+1} = x_k + alpha d_k: dL/dd_k = alpha dL/dx_{k+1}; dL/dx_k = dL/dx_{k+1} - sbar_k
    for (int e = T.rank(); e < len; e += T.size()) aw.DB[e] = alpha * aw.XB[e];
    if (fl & kTapeKept) tvaxpy(T, aw.XB, -1.0, aw.sbar + (size_t)k * len, len);
    T.sync();
    // (4) d_k = -H_k g_k: active pairs at iteration k (newest first)
    int plist[kHistory];
    int h = 0;
    if (!(fl & kTapeReset)) {
      int ring[kHistory];
      int cnt = 0;
      for (int j = 0; j < k; ++j) {
        if (aw.tape.flags[j] & kTapeReset) cnt = 0;
        if (aw.tape.flags[j] & kTapeKept) {
          if (cnt < kHistory) {
            ring[cnt++] = j;
          } else {
            for (int q = 0; q + 1 < kHistory; ++q) ring[q] = ring[q + 1];
            ring[kHistory - 1] = j;
          }
        }
      }
      h = cnt;
      for (int q = 0; q < h; ++q) plist[q] = ring[h - 1 - q];
    }
    // forward recompute of the two-loop with intermediates: Qs[t] before pair plist[t]
    double acoef[kHistory], bcoef[kHistory], abar[kHistory];
    const double* gk = tG + (size_t)k * len;
    for (int e = T.rank(); e < len; e += T.size()) aw.Qs[e] = gk[e];
    T.sync();
    for (int t = 0; t < h; ++t) {
      const int i = plist[t];
      const double* si = aw.sP + (size_t)i * len;
      const double* yi = aw.yP + (size_t)i * len;
      double* qt = aw.Qs + (size_t)t * len;
      double* qn = aw.Qs + (size_t)(t + 1) * len;
      acoef[t] = aw.rho[i] * tdot(T, si, qt, len);
      for (int e = T.rank(); e < len; e += T.size()) qn[e] = qt[e] - acoef[t] * yi[e];
      T.sync();
      abar[t] = 0.0;
    }
    team_solve(T, ty, w, P, aw.Qs + (size_t)h * len, aw.Rs);
    for (int u = 0; u < h; ++u) {
      const int t = h - 1 - u, i = plist[t];
      const double* si = aw.sP + (size_t)i * len;
      const double* yi = aw.yP + (size_t)i * len;
      const double* ru = aw.Rs + (size_t)u * len;
      double* rn = aw.Rs + (size_t)(u + 1) * len;
      bcoef[u] = aw.rho[i] * tdot(T, yi, ru, len);
      const double c = acoef[t] - bcoef[u];
      for (int e = T.rank(); e < len; e += T.size()) rn[e] = ru[e] + c * si[e];
      T.sync();
    }
    // reverse: dL/dr_h = -dL/dd_k
    for (int e = T.rank(); e < len; e += T.size()) aw.RB[e] = -aw.DB[e];
    for (int q = 0; q < h; ++q)
      if (T.leader()) aw.rhobar[plist[q]] = 0.0;
    T.sync();
    for (int u = h - 1; u >= 0; --u) {
      const int t = h - 1 - u, i = plist[t];
      const double* si = aw.sP + (size_t)i * len;
      const double* yi = aw.yP + (size_t)i * len;
      const double* ru = aw.Rs + (size_t)u * len;
      const double c = acoef[t] - bcoef[u];
      const double cb = tdot64(T, aw.RB, si, len);
      const double yr = tdot64(T, yi, ru, len);
      tvaxpy(T, aw.sbar + (size_t)i * len, c, aw.RB, len);
      abar[t] += cb;
      const double bb = -cb;
      if (T.leader()) aw.rhobar[i] += bb * yr;
      tvaxpy(T, aw.ybar + (size_t)i * len, bb * aw.rho[i], ru, len);
      tvaxpy(T, aw.RB, bb * aw.rho[i], yi, len);
      T.sync();
    }
    // r_0 = A^-1 q_h: dL/dq_h = A^-1 dL/dr_0; dL/dw via dA/dw (A carries the elastic part
    // L as (1 + c_beta/dt) L under Rayleigh damping)
    team_solve(T, ty, w, P, aw.RB, aw.QB);
    {
      double fs, fb;
      matrix_weight_forms(ty, aw.QB, aw.Rs, &fs, &fb, T);
      wacc[0] -= (1.0 + ty.damp_l) * fs;
      wacc[1] -= (1.0 + ty.damp_l) * fb;
    }
    for (int t = h - 1; t >= 0; --t) {
      const int i = plist[t];
      const double* si = aw.sP + (size_t)i * len;
      const double* yi = aw.yP + (size_t)i * len;
      const double* qt = aw.Qs + (size_t)t * len;
      abar[t] -= tdot64(T, yi, aw.QB, len);
      const double sq = tdot64(T, si, qt, len);
      tvaxpy(T, aw.ybar + (size_t)i * len, -acoef[t], aw.QB, len);
      if (T.leader()) aw.rhobar[i] += abar[t] * sq;
      tvaxpy(T, aw.sbar + (size_t)i * len, abar[t] * aw.rho[i], qt, len);
      tvaxpy(T, aw.QB, abar[t] * aw.rho[i], si, len);
      T.sync();
    }
    tvaxpy(T, gbk, 1.0, aw.QB, len);
    T.sync();
    // rho_i = 1/(y_i . s_i)
    for (int t = 0; t < h; ++t) {
      const int i = plist[t];
      const double r2 = aw.rho[i] * aw.rho[i] * aw.rhobar[i];
      tvaxpy(T, aw.ybar + (size_t)i * len, -r2, aw.sP + (size_t)i * len, len);
      tvaxpy(T, aw.sbar + (size_t)i * len, -r2, aw.yP + (size_t)i * len, len);
    }
    T.sync();
  }
  // g_0 = grad f(x_0)
  hessian_vector(ty, w, tU, aw.gbar, aw.HV, cvol, wd, T);
  for (int q = 0; q < 4; ++q) wacc[q] += wd[q];
  // Rayleigh damping: every g_k holds C (x_k - x_n) / dt, so dL/dx_n gains
  // -C/dt times the sum of all gradient adjoints (into RB, summed in DB)
  const bool damped = ty.damp_m != 0.0 || ty.damp_l != 0.0;
  if (damped) {
    for (int e = T.rank(); e < len; e += T.size()) {
      double sg = 0.0;
      for (int k = 0; k <= K; ++k) sg += aw.gbar[(size_t)k * len + e];
      aw.DB[e] = sg;
    }
    T.sync();
    apply_rayleigh(ty, w, aw.DB, aw.RB, T);
  }
  // x_0 = y; y = x_n + dt v_n + dt^2 M^-1 f;  v_{n+1} = (x_K - x_n)/dt
  for (int vtx = T.rank(); vtx < n; vtx += T.size()) {
    const double mi = __ldg(&ty.mass[vtx]);
    for (int c = 0; c < 3; ++c) {
      const int e = 3 * vtx + c;
      const double yb = aw.YB[e] - mi / (dt * dt) * aw.gbar[e] + aw.XB[e] + aw.HV[e];
      const double gvv = A.gv_next ? A.gv_next[c * Nt + off + vtx] : 0.0;
      A.gx[c * Nt + off + vtx] = yb - gvv / dt - (damped ? aw.RB[e] : 0.0);
      A.gv[c * Nt + off + vtx] = dt * yb;
      A.gf[c * Nt + off + vtx] = dt * dt / mi * yb;
    }
  }
  if (T.leader())
    for (int q = 0; q < 4; ++q) A.gw[(size_t)cell * 4 + q] = wacc[q];
  T.sync();
}

// The unrolled adjoint, one CTA of kAdjWarps warps per cell (work queue over the cells).
// Warp 0 recomputes the forward step with the tape (the warp-level fused step, whose
// iterates are the FP64 split step's bit for bit) and runs the warp-level FP64 solves;
// the reverse sweep's vector passes, Hessian-vector products and sums use the whole CTA
// (a warp per cell kept the FP64 pipe about 20 % busy: each warp waits on its memory).
// Each CTA uses one workspace slot and one solve vector in shared memory.
constexpr int kAdjWarps = 4;
__global__ void __launch_bounds__(32 * kAdjWarps) npfem_adjoint_kernel(DevTypeView<double> ty, StepParams P,
                                                                       AdjParams A, const double* x,
                                                                       const double* v, const double* f) {
  extern __shared__ double smem_z[];
  __shared__ CtaShared sh;
  int par = 0;
  const int lane = threadIdx.x & 31;
  const int slot = blockIdx.x;
  double* zs = P.z_in_smem ? smem_z : nullptr;
  CellWs<double> w = carve<double>(P.scratch + (size_t)slot * P.slot_bytes, ty.n, ty.T, ty.E, zs);
  AdjWs aw = carve_adj(A.scratch + (size_t)slot * A.slot_bytes, ty.n);
  const CtaTeam team{&sh, &par};
  for (;;) {
    if (threadIdx.x == 0) sh.item = atomicAdd(P.queue_counter, 1);
    __syncthreads();
    const int item = sh.item;
    __syncthreads();
    if (item >= P.ncells_list) break;
    const int cell = P.cell_list[item];
    const int iters = P.iters ? P.iters[cell] : P.iters_default;
    if (iters < 0 || iters > kMaxAdjIters) {  // the same for the whole CTA
      if (threadIdx.x == 0 && P.status_out) P.status_out[cell] = 8;
      continue;
    }
    if (threadIdx.x < 32)
      process_cell<double, true>(ty, P, w, cell, const_cast<double*>(x), const_cast<double*>(v), f, lane, &aw.tape);
    __syncthreads();
    reverse_cell(ty, P, A, w, aw, cell, iters, team);
    if (threadIdx.x == 0 && P.status_out) P.status_out[cell] = 0;
  }
}

// out = C a / dt = (c_alpha/dt) M a + (c_beta/dt) L a (Rayleigh damping), through the
// element buffers and the gradient gather of the step.
template <class Tm>
__device__ void apply_rayleigh(const DevTypeView<double>& ty, const CellWs<double>& w, const double* a,
                               double* out, const Tm& T) {
  const int n = ty.n;
  for (int i = T.rank(); i < 9 * ty.T; i += T.size()) w.corner[i] = 0.0;
  for (int i = T.rank(); i < 3 * ty.E; i += T.size()) w.hbuf[i] = 0.0;
  T.sync();
  if (ty.damp_l != 0.0 && T.solver())
    damping_elastic<double>(ty.tris, ty.Dinv, ty.w_tri, ty.hinges, ty.c_hinge, ty.w_hinge, ty.T, ty.E, ty.damp_l,
                            a, w.corner, w.hbuf, T.lane());
  T.sync();
  for (int vtx = T.rank(); vtx < n; vtx += T.size()) {
    V3<double> g = (ty.damp_m * __ldg(&ty.mass[vtx])) * ld3(a, vtx);
    const int e0 = __ldg(&ty.inc_ptr[vtx]), e1 = __ldg(&ty.inc_ptr[vtx + 1]);
    for (int e = e0; e < e1; ++e) {
      const int code = __ldg(&ty.inc_code[e]);
      if (code >= 0)
        g = g + ld3(w.corner, code);
      else
        g = g + __ldg(&ty.inc_coef[e]) * ld3(w.hbuf, (-code - 1) >> 2);
    }
    st3(out, vtx, g);
  }
  T.sync();
}

// ------------------------------------------------------------------ implicit adjoint
// Gradients through the converged minimiser x* of the step objective (the solver run to
// convergence, Implementation and architecture section) by the implicit-function
// theorem: grad f(x*; y, w) = 0, so with H = grad^2 f(x*)
//   H lam = dL/dx* + dL/dv*/dt   (v* = (x* - x_n)/dt),
//   dL/dy = (M/dt^2) lam,  dL/dx_n = dL/dy - dL/dv*/dt,  dL/dv_n = dt dL/dy,
//   dL/df = lam,  dL/dw_q = -lam . d(grad f)/dw_q,
// and with Rayleigh damping, whose dissipation term depends on x_n directly, dL/dx_n gains
// C lam / dt (the Hessian and the weight terms include the damping already).
// lam comes from conjugate gradients on H (Hessian-vector products), preconditioned by
// the prefactored projective-dynamics matrix A^-1; the forward step that produced x* is
// the caller's (npfem_step on copies of the inputs).
struct ImplicitParams {
  const double* x_n;      // [3][Nt] the step's input positions
  const double* x_star;   // [3][Nt] the converged positions
  const double* gx_next;  // [3][Nt] dL/dx*
  const double* gv_next;  // [3][Nt] dL/dv* or null
  double* gx;             // [3][Nt] out
  double* gv;
  double* gf;
  double* gw;             // [ncells][4] out
  char* scratch;          // 6 [3n] FP64 vectors per warp slot
  size_t slot_bytes;
  double cg_tol;          // stop when |r| <= cg_tol |b|
  int cg_max;
  int32_t* status_out;    // [ncells] or null: bit 16 ORed in when CG did not converge
};

constexpr int kImplicitVectors = 6;
constexpr int kStatusCgNotConverged = 16;

__global__ void __launch_bounds__(128) npfem_adjoint_implicit_kernel(DevTypeView<double> ty, StepParams P,
                                                                      ImplicitParams A) {
  extern __shared__ double smem_z[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int slot = blockIdx.x * (blockDim.x >> 5) + wib;
  double* zs = P.z_in_smem ? smem_z + (size_t)wib * (P.solve_per_coord ? 1 : 3) * (ty.n + 1) : nullptr;
  CellWs<double> w = carve<double>(P.scratch + (size_t)slot * P.slot_bytes, ty.n, ty.T, ty.E, zs);
  const int n = ty.n, len = 3 * n;
  double* lam = reinterpret_cast<double*>(A.scratch + (size_t)slot * A.slot_bytes);
  double* r = lam + len;
  double* z = r + len;
  double* pv = z + len;
  double* hp = pv + len;
  double* U = hp + len;
  const int64_t Nt = P.n_total;
  const double dt = ty.dt;
  for (;;) {
    int item = 0;
    if (lane == 0) item = atomicAdd(P.queue_counter, 1);
    item = __shfl_sync(kFull, item, 0);
    if (item >= P.ncells_list) break;
    const int cell = P.cell_list[item];
    const int64_t off = P.offsets[cell];
    const double ax = A.x_n[off], ay = A.x_n[Nt + off], az = A.x_n[2 * Nt + off];
    Acc<double> cx, cy, cz, bb;
    for (int k = lane; k < n; k += 32) {
      const double anc[3] = {ax, ay, az};
      for (int c = 0; c < 3; ++c) {
        const double xn = A.x_n[c * Nt + off + k];
        w.X[3 * k + c] = xn - anc[c];
        U[3 * k + c] = A.x_star[c * Nt + off + k] - xn;
        const double gvv = A.gv_next ? A.gv_next[c * Nt + off + k] : 0.0;
        const double b = A.gx_next[c * Nt + off + k] + gvv / dt;
        r[3 * k + c] = b;
        lam[3 * k + c] = 0.0;
        bb.add_prod(b, b);
      }
      cx.add(w.X[3 * k]);
      cy.add(w.X[3 * k + 1]);
      cz.add(w.X[3 * k + 2]);
    }
    const V3<double> cvol{cx.total() / n, cy.total() / n, cz.total() / n};
    const double bn = sqrt(bb.total());
    __syncwarp();
    bool converged = bn == 0.0;
    double wd[4];
    if (!converged) {
      global_solve<double>(ty, w.z, P.z_in_smem != 0, r, z, lane, P.solve_per_coord != 0);
      for (int e = lane; e < len; e += 32) pv[e] = z[e];
      __syncwarp();
      double rz = vdot64<double>(r, z, len, lane);
      for (int it = 0; it < A.cg_max; ++it) {
        hessian_vector(ty, w, U, pv, hp, cvol, wd, WarpTeam{lane});
        const double php = vdot64<double>(pv, hp, len, lane);
        if (!(php > 0.0)) break;  // not positive definite along p: stop, report
        const double a = rz / php;
        vaxpy(lam, a, pv, len, lane);
        vaxpy(r, -a, hp, len, lane);
        __syncwarp();
        const double rn = sqrt(vdot64<double>(r, r, len, lane));
        if (rn <= A.cg_tol * bn) {
          converged = true;
          break;
        }
        global_solve<double>(ty, w.z, P.z_in_smem != 0, r, z, lane, P.solve_per_coord != 0);
        const double rz1 = vdot64<double>(r, z, len, lane);
        const double beta = rz1 / rz;
        rz = rz1;
        for (int e = lane; e < len; e += 32) pv[e] = z[e] + beta * pv[e];
        __syncwarp();
      }
    }
    // weight derivatives: wd[q] = lam . d(grad f)/d(w_q)
    hessian_vector(ty, w, U, lam, hp, cvol, wd, WarpTeam{lane});
    const bool damped = ty.damp_m != 0.0 || ty.damp_l != 0.0;
    if (damped) apply_rayleigh(ty, w, lam, z, WarpTeam{lane});  // z <- C lam / dt
    for (int vtx = lane; vtx < n; vtx += 32) {
      const double mi = __ldg(&ty.mass[vtx]);
      for (int c = 0; c < 3; ++c) {
        const double l = lam[3 * vtx + c];
        const double dldy = mi / (dt * dt) * l;
        const double gvv = A.gv_next ? A.gv_next[c * Nt + off + vtx] : 0.0;
        A.gx[c * Nt + off + vtx] = dldy - gvv / dt + (damped ? z[3 * vtx + c] : 0.0);
        A.gv[c * Nt + off + vtx] = dt * dldy;
        A.gf[c * Nt + off + vtx] = l;
      }
    }
    if (lane == 0) {
      for (int q = 0; q < 4; ++q) A.gw[(size_t)cell * 4 + q] = -wd[q];
      if (A.status_out && !converged) A.status_out[cell] |= kStatusCgNotConverged;
    }
    __syncwarp();
  }
}

}  // namespace npfem
