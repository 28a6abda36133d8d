// Internal data structures of the npFEM library (host setup <-> CUDA kernels).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace npfem {

constexpr int kHistory = 5;              // L-BFGS pairs kept (m)
constexpr int kMaxHalvings = 20;         // line-search backtracking limit
constexpr double kArmijoC1 = 1e-4;
constexpr double kEnergyGuardEps = 1e-6; // approximate-Armijo energy guard (relative)
constexpr double kCurvatureEps = 1e-12;  // keep pair only if s.y > eps |s||y|
constexpr double kDegenerateDet = 1e-30; // det(F^T F) below this: triangle skipped
constexpr double kDegenerateNorm = 1e-30;
constexpr int kChunk = 32;               // entries per triangular-solve chunk (one per lane)
constexpr int kCtaPacks = 4;             // level packings for CTA-cooperative sweeps
constexpr int kCtaWarps[kCtaPacks] = {2, 4, 6, 8};
constexpr int kMaxColours = 64;          // colour classes of triangles or of hinges
// Warps per cell of the FP32 form's default CTA iteration kernels for an n-vertex type
// (its colour classes are balanced for that CTA size).
inline int default_cta_warps(int n) { return n <= 256 ? 2 : (n <= 1024 ? 4 : 8); }

// Host-side result of the per-type setup (all FP64; the device upload makes FP32
// copies of the element constants for the FP32-form kernels).
struct HostType {
  int n = 0, T = 0, E = 0;
  std::vector<int32_t> tris;     // [T][3]
  std::vector<double> Dinv;      // [T][3] (d00, d01, d11) of the upper-triangular Dm^-1
  std::vector<double> w_tri;     // [T]
  std::vector<double> area;      // [T] rest areas
  std::vector<int32_t> hinges;   // [E][4] (i, j, kA, kB)
  // Elements are stored colour by colour: no two triangles (hinges) of one colour share a
  // vertex; colour c holds [cptr[c], cptr[c+1]).  Empty when more than kMaxColours
  // colours would be needed (the CTA iteration kernels are then not used for the type).
  std::vector<int32_t> tri_cptr, hinge_cptr;
  std::vector<double> c_hinge;   // [E][4]
  std::vector<double> K0;        // [E][4] (K0x, K0y, K0z, |K0|)
  std::vector<double> w_hinge;   // [E]
  std::vector<double> hinge_unit;  // [E] 3/(A_A+A_B): w_hinge per unit bending weight
  std::vector<double> mass;      // [n]
  double A0 = 0, V0 = 0, w_area = 0, w_vol = 0, dt = 0, total_mass = 0;
  double c_alpha = 0, c_beta = 0;  // Rayleigh damping
  double s_min = 1, s_max = 1;     // strain limits (singular values of F clamped to them)
  // gradient gather: per vertex, corner codes (t*3+slot >= 0) and hinge codes
  // (-(h*4+k)-1 < 0) with the hinge coefficient
  std::vector<int32_t> inc_ptr;  // [n+1]
  std::vector<int32_t> inc_code; // [nnz]
  std::vector<double> inc_coef;  // [nnz]
  // global solve: A = P^T Lt D Lt^T P with unit lower Lt; row r of the factor is vertex perm[r]
  std::vector<int32_t> perm;     // [n]
  std::vector<double> dinv;      // [n] 1/D
  int64_t nnz_factor = 0;
  // Triangular sweeps as chunks of 32 updates z[row] -= val * z[col], one per lane
  // (padding: row = col = n, val = 0).  meta bit 0: synchronise the warp before the
  // chunk (it reads or writes a row written since the last synchronisation).
  std::vector<int32_t> fwd_meta, bwd_meta;   // [nchunks]
  std::vector<uint32_t> fwd_rc, bwd_rc;      // [nchunks*32] row | col << 16
  std::vector<double> fwd_val, bwd_val;      // [nchunks*32]
  // The same sweeps packed for a CTA of W warps that sweeps one cell together: levels
  // of W sub-chunks of 32 updates (sub-chunk w of level L at [L*W + w]); the targets of
  // a level are distinct.  meta[L*W + w] bit 0: barrier of the CTA before level L (it
  // reads or writes a row written since the last barrier; equal for all w); bit 1:
  // sub-chunk w of level L is empty.
  struct LevelPack {
    int W = 0;
    std::vector<int32_t> fwd_meta, bwd_meta;   // [nlevels*W]
    std::vector<uint32_t> fwd_rc, bwd_rc;      // [nlevels*W*32]
    std::vector<double> fwd_val, bwd_val;      // [nlevels*W*32]
  };
  LevelPack cta[kCtaPacks];                    // W = kCtaWarps[i]
};

// One update of a triangular sweep: z[t] -= v * z[s], valid once every update that
// targets s has been applied.  Indices satisfy t > s (in the sweep's own order).
struct SweepOp {
  int t, s;
  double v;
};

// Pack the updates of one sweep into levels of W x 32 updates (relabel maps r -> n-1-r
// when emitting indices); see HostType for the layout.
void pack_sweep(int n, const std::vector<SweepOp>& ops, bool relabel, int W, std::vector<int32_t>* meta,
                std::vector<uint32_t>* rc, std::vector<double>* val);

// Build the host type.  Returns 0 or a negative NPFEM_ERR_* code with a message.
int build_host_type(int n, int T, const double* xyz, const int32_t* tris, double w_strain,
                    double w_bend, double w_area, double w_vol, double density, double dt,
                    double c_alpha, double c_beta, HostType* out, std::string* err);

// ------------------------------------------------------------------ device view
template <typename S>
struct DevTypeView {
  int n, T, E;
  int nchunks_fwd, nchunks_bwd;
  int cta_nlev_fwd[kCtaPacks], cta_nlev_bwd[kCtaPacks];   // levels of the CTA packings
  const int32_t* tris;      // [T][3]
  const int32_t* tri4;      // [T][4] (i0, i1, i2, 0): one 16-byte load per triangle
  const S* trc;             // [T][4] (d00, d01, d11, w_tri): one vector load per triangle
  const S* Dinv;            // [T][3]
  const S* w_tri;           // [T]
  const int32_t* hinges;    // [E][4]
  const S* c_hinge;         // [E][4]
  const S* K0;              // [E][4]
  const S* w_hinge;         // [E]
  const S* tri_area;        // [T] rest areas (w_tri per unit strain weight)
  const S* hinge_unit;      // [E] w_hinge per unit bending weight
  const S* mass;            // [n]
  const S* inv_mass;        // [n]
  const int32_t* inc_ptr;   // [n+1]
  const int32_t* inc_code;  // [nnz]
  const S* inc_coef;        // [nnz]
  const int32_t* perm;      // [n]
  const double* dinv;       // [n]
  const int32_t* fwd_meta;
  const uint32_t* fwd_rc;
  const double* fwd_val;
  const int32_t* bwd_meta;
  const uint32_t* bwd_rc;
  const double* bwd_val;
  const int32_t* cta_fwd_meta[kCtaPacks];
  const uint32_t* cta_fwd_rc[kCtaPacks];
  const double* cta_fwd_val[kCtaPacks];
  const int32_t* cta_bwd_meta[kCtaPacks];
  const uint32_t* cta_bwd_rc[kCtaPacks];
  const double* cta_bwd_val[kCtaPacks];
  double A0, V0, w_area, w_vol, dt;
  double inv_A0, inv_V0, idt2, inv_dt, inv_n;  // 1 / A0, 1 / V0, 1 / dt^2, 1 / dt, 1 / n
  double damp_m, damp_l;    // Rayleigh damping over dt: c_alpha/dt (mass part), c_beta/dt (elastic part)
  double s_min, s_max;      // strain limits; limited = 0 for the rotations [1, 1]
  int limited;
  int ntc, nhc;             // colour classes of the triangles and hinges (0: not coloured)
  const int32_t* tri_cptr;  // [ntc+1] first triangle of each colour
  const int32_t* hinge_cptr;  // [nhc+1] first hinge of each colour
};

}  // namespace npfem
