// Contact detection at the start of a step (collision reading): every vertex i of cell a
// is matched with the nearest vertex j of each other cell b closer than the search
// radius, and the two nearest such cells are kept (nearest first; equal distances: the
// smaller j within a cell, the smaller b across cells).  Each match becomes a plane
// through x_j with the unit area-weighted outward normal n_j of b, fixed for the step;
// the step objective adds (w/2) max(0, delta - (n_j . x_i - n_j . x_j))^2 per match.
// The paper names collision detection, collision forces and a collision weight
// (Performance figure, "Other"; Collision at an obstacle section) and uses them to pack
// randomly placed cells without fluid (Cell Packing section); it prints no formula.
//
// Pipeline (all on the step's stream, graph-capturable):
//   k_normals  per cell: n_i = normalise(sum over incident triangles (x1-x0) x (x2-x0))
//   k_hash     per vertex: grid cell (edge = radius) -> bucket of a power-of-two hash table
//   k_scan_*   exclusive prefix sum of the bucket counts (block scan, carry scan, add)
//   k_scatter  vertices into bucket order, with their position (float) and cell index
//   k_query    per vertex: the 27 neighbouring grid cells; squared distances in float,
//              with a bound m on their difference from the FP64 value (from the largest
//              coordinate magnitude, gathered by k_hash); a decision (inside the radius,
//              nearer than another candidate) is taken in float when the float values
//              are more than m apart, and otherwise from the exact FP64 squared distance,
//              evaluated as (dx*dx + dy*dy) + dz*dz without contraction -- so every
//              decision is the one an FP64 evaluation in that order takes
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "npfem_internal.h"

namespace npfem {

constexpr int kContactSlots = 2;
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 4;
constexpr int kScanBlock = kScanThreads * kScanPerThread;

struct ContactParams {
  int64_t n_total;
  const int32_t* vcell;      // [N] cell of each vertex
  const int64_t* offsets;    // [ncells+1]
  double h, h_inv, r2;       // grid edge (= radius), its inverse, radius^2
  uint32_t mask;             // hash table size - 1
  int32_t* key;              // [N] bucket of each vertex
  int32_t* count;            // [T] bucket counts
  int32_t* start;            // [T+1] bucket starts (exclusive scan)
  int32_t* cursor;           // [T] scatter cursors
  int32_t* bsum;             // [T / kScanBlock] block sums
  int32_t* sorted;           // [N] vertex ids in bucket order
  float4* sortpos;           // [N] position (float) + cell id, bucket order
  int32_t* maxabs;           // [1] largest |coordinate| of the step's input (float bits)
  double* box;               // [6] wall box lo, hi (collisions with walls)
  double* nrm;               // [N][3] unit vertex normals
  int32_t* ccount;           // [N] matches per vertex (0..2)
  int32_t* cvertex;          // [N][2] matched vertex (-1: unused)
  double* cplane;            // [N][2][4] normal, offset n . (x_j - x_anchor(cell of i))
};

__device__ __forceinline__ int grid_coord(double v, double h_inv) { return (int)floor(v * h_inv); }

__device__ __forceinline__ uint32_t grid_hash(int ix, int iy, int iz, uint32_t mask) {
  return (((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^ ((uint32_t)iz * 83492791u)) & mask;
}

// Unit area-weighted vertex normals of the cells of one type, one CTA per cell: the
// triangles' cross products (x1-x0) x (x2-x0) once into shared memory ([T][3] FP64),
// then per vertex their sum over its incident triangles, in triangle order (the order of
// the corner codes in the gradient gather's incidence list), normalised.
template <typename S>
__global__ void __launch_bounds__(128) npfem_k_normals(DevTypeView<S> ty, const int32_t* cells, int ncells,
                                                       const int64_t* offsets, int64_t Nt, const S* x, double* nrm) {
  extern __shared__ double tri_n[];
  for (int c = blockIdx.x; c < ncells; c += gridDim.x) {
    const int64_t off = offsets[cells[c]];
    for (int t = threadIdx.x; t < ty.T; t += blockDim.x) {
      const int64_t i0 = off + __ldg(&ty.tris[3 * t]), i1 = off + __ldg(&ty.tris[3 * t + 1]),
                    i2 = off + __ldg(&ty.tris[3 * t + 2]);
      const double ax = (double)x[i1] - (double)x[i0], ay = (double)x[Nt + i1] - (double)x[Nt + i0],
                   az = (double)x[2 * Nt + i1] - (double)x[2 * Nt + i0];
      const double bx = (double)x[i2] - (double)x[i0], by = (double)x[Nt + i2] - (double)x[Nt + i0],
                   bz = (double)x[2 * Nt + i2] - (double)x[2 * Nt + i0];
      tri_n[3 * t] = ay * bz - az * by;
      tri_n[3 * t + 1] = az * bx - ax * bz;
      tri_n[3 * t + 2] = ax * by - ay * bx;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < ty.n; v += blockDim.x) {
      double sx = 0.0, sy = 0.0, sz = 0.0;
      const int e0 = __ldg(&ty.inc_ptr[v]), e1 = __ldg(&ty.inc_ptr[v + 1]);
      for (int e = e0; e < e1; ++e) {
        const int code = __ldg(&ty.inc_code[e]);
        if (code < 0) continue;
        const int t = code / 3;
        sx += tri_n[3 * t];
        sy += tri_n[3 * t + 1];
        sz += tri_n[3 * t + 2];
      }
      const double inv = 1.0 / sqrt(sx * sx + sy * sy + sz * sz);
      double* o = nrm + 3 * (off + v);
      o[0] = sx * inv;
      o[1] = sy * inv;
      o[2] = sz * inv;
    }
    __syncthreads();
  }
}

template <typename S>
__global__ void npfem_k_hash(ContactParams C, const S* x) {
  const int64_t Nt = C.n_total;
  float amax = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nt; i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = grid_coord((double)x[i], C.h_inv), iy = grid_coord((double)x[Nt + i], C.h_inv),
              iz = grid_coord((double)x[2 * Nt + i], C.h_inv);
    const uint32_t k = grid_hash(ix, iy, iz, C.mask);
    C.key[i] = (int32_t)k;
    atomicAdd(&C.count[k], 1);
    amax = fmaxf(amax, fmaxf(fabsf((float)x[i]), fmaxf(fabsf((float)x[Nt + i]), fabsf((float)x[2 * Nt + i]))));
  }
  // non-negative floats order like their bit patterns: one integer maximum per warp
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if ((threadIdx.x & 31) == 0) atomicMax(C.maxabs, __float_as_int(amax));
}

// Exclusive scan within blocks of kScanBlock entries; block totals to bsum.
__global__ void __launch_bounds__(kScanThreads) npfem_k_scan_blocks(const int32_t* in, int32_t* out, int32_t* bsum) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)tid * kScanPerThread;
  int32_t v[kScanPerThread];
  int32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    v[k] = in[base + k];
    s += v[k];
  }
  int32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    int32_t t = warp_tot[lane];
    int32_t ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += u;
    }
    warp_tot[lane] = ti - t;  // exclusive prefix of the warp totals
    if (lane == 31) bsum[blockIdx.x] = ti;
  }
  __syncthreads();
  int32_t run = warp_tot[w] + incl - s;
#pragma unroll
  for (int k = 0; k < kScanPerThread; ++k) {
    out[base + k] = run;
    run += v[k];
  }
}

// Exclusive scan of the block totals in place (one block, chunks of kScanBlock with a carry).
__global__ void __launch_bounds__(kScanThreads) npfem_k_scan_carry(int32_t* bsum, int nblocks) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  __shared__ int32_t carry;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 < nblocks; c0 += kScanBlock) {
    int32_t v[kScanPerThread];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
      const int idx = c0 + tid * kScanPerThread + k;
      v[k] = idx < nblocks ? bsum[idx] : 0;
      s += v[k];
    }
    int32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    int32_t chunk_total = 0;
    if (w == 0) {
      int32_t t = warp_tot[lane];
      int32_t ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += u;
      }
      warp_tot[lane] = ti - t;
      chunk_total = __shfl_sync(0xffffffffu, ti, 31);
    }
    __syncthreads();
    int32_t run = carry + warp_tot[w] + incl - s;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
      const int idx = c0 + tid * kScanPerThread + k;
      if (idx < nblocks) bsum[idx] = run;
      run += v[k];
    }
    __syncthreads();
    if (tid == 0) carry += chunk_total;
    __syncthreads();
  }
}

// start[i] += scanned block total; cursor = start; start[T] = N.
__global__ void npfem_k_scan_add(ContactParams C, int64_t T) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t s = C.start[i] + C.bsum[i / kScanBlock];
    C.start[i] = s;
    C.cursor[i] = s;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) C.start[T] = (int32_t)C.n_total;
}

template <typename S>
__global__ void npfem_k_scatter(ContactParams C, const S* x) {
  const int64_t Nt = C.n_total;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nt; i += (int64_t)gridDim.x * blockDim.x) {
    const int pos = atomicAdd(&C.cursor[C.key[i]], 1);
    C.sorted[pos] = (int32_t)i;
    C.sortpos[pos] = make_float4((float)x[i], (float)x[Nt + i], (float)x[2 * Nt + i], __int_as_float(C.vcell[i]));
  }
}

struct Match {
  float d2f;  // float squared distance
  int b, j;   // cell, vertex (j < 0: empty slot)
};

// Exact FP64 squared distance from (px, py, pz) to vertex j, rounded operation by operation.
template <typename S>
__device__ __forceinline__ double exact_d2(const S* x, int64_t Nt, double px, double py, double pz, int j) {
  const double dx = px - (double)x[j], dy = py - (double)x[Nt + j], dz = pz - (double)x[2 * Nt + j];
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Is candidate (df, j) before slot s in the order (d2, key)?  key is the vertex index
// within one cell and the cell index across cells.  Float decides when the float values
// are more than m apart (they are then ordered like the FP64 values); otherwise both
// exact FP64 distances are compared.
template <typename S>
__device__ __forceinline__ bool before(float df, int j, int key, const Match& s, int skey, float m, const S* x,
                                       int64_t Nt, double px, double py, double pz) {
  if (s.j < 0) return true;
  if (df < s.d2f - m) return true;
  if (df > s.d2f + m) return false;
  const double dj = exact_d2(x, Nt, px, py, pz, j), ds = exact_d2(x, Nt, px, py, pz, s.j);
  return dj < ds || (dj == ds && key < skey);
}

template <typename S>
__device__ __forceinline__ void offer(Match* s, float df, int b, int j, float m, const S* x, int64_t Nt, double px,
                                      double py, double pz) {
  if (b == s[0].b || b == s[1].b) {
    Match& t = b == s[0].b ? s[0] : s[1];
    if (before(df, j, j, t, t.j, m, x, Nt, px, py, pz)) {
      t.d2f = df;
      t.j = j;
    }
  } else if (before(df, j, b, s[1], s[1].b, m, x, Nt, px, py, pz)) {
    s[1] = Match{df, b, j};
  }
  if (s[1].j >= 0 && before(s[1].d2f, s[1].j, s[1].b, s[0], s[0].b, m, x, Nt, px, py, pz)) {
    const Match t = s[0];
    s[0] = s[1];
    s[1] = t;
  }
}

template <typename S>
__global__ void __launch_bounds__(128) npfem_k_query(ContactParams C, const S* x) {
  const int64_t Nt = C.n_total;
  // bound on |float d2 - FP64 d2| for candidates within ~r: each coordinate is rounded to
  // float (error <= u M, u = 2^-24, M the largest magnitude), the difference and the
  // squares and sums add a few u r^2; a factor two of slack on top
  const double u = 1.0 / 16777216.0;
  const double r = sqrt(C.r2);
  const double M = (double)__int_as_float(*C.maxabs);
  const float m = (float)(2.0 * (16.0 * u * r * (M + r) + 8.0 * u * C.r2));
  const float r2f = (float)C.r2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nt; i += (int64_t)gridDim.x * blockDim.x) {
    const int a = C.vcell[i];
    const double px = (double)x[i], py = (double)x[Nt + i], pz = (double)x[2 * Nt + i];
    const int ix = grid_coord(px, C.h_inv), iy = grid_coord(py, C.h_inv), iz = grid_coord(pz, C.h_inv);
    const float xf = (float)x[i], yf = (float)x[Nt + i], zf = (float)x[2 * Nt + i];
    Match s[kContactSlots] = {{0.f, 0x7fffffff, -1}, {0.f, 0x7fffffff, -1}};
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          const uint32_t k = grid_hash(ix + ox, iy + oy, iz + oz, C.mask);
          const int q1 = C.start[k + 1];
          for (int q = C.start[k]; q < q1; ++q) {
            const float4 sp = C.sortpos[q];
            const int b = __float_as_int(sp.w);
            if (b == a) continue;
            const float fx = sp.x - xf, fy = sp.y - yf, fz = sp.z - zf;
            const float df = fx * fx + fy * fy + fz * fz;
            if (df > r2f + m) continue;
            const int j = C.sorted[q];
            if (df >= r2f - m && !(exact_d2(x, Nt, px, py, pz, j) < C.r2)) continue;
            offer(s, df, b, j, m, x, Nt, px, py, pz);
          }
        }
    const int64_t anc = C.offsets[a];
    const double axx = (double)x[anc], ayy = (double)x[Nt + anc], azz = (double)x[2 * Nt + anc];
    int cnt = 0;
#pragma unroll
    for (int mm = 0; mm < kContactSlots; ++mm) {
      double* pl = C.cplane + 8 * i + 4 * mm;
      if (s[mm].j >= 0) {
        const int j = s[mm].j;
        const double nx = C.nrm[3 * j], ny = C.nrm[3 * j + 1], nz = C.nrm[3 * j + 2];
        pl[0] = nx;
        pl[1] = ny;
        pl[2] = nz;
        pl[3] = nx * ((double)x[j] - axx) + ny * ((double)x[Nt + j] - ayy) + nz * ((double)x[2 * Nt + j] - azz);
        C.cvertex[2 * i + mm] = j;
        cnt = mm + 1;
      } else {
        pl[0] = pl[1] = pl[2] = pl[3] = 0.0;
        C.cvertex[2 * i + mm] = -1;
      }
    }
    C.ccount[i] = cnt;
  }
}

}  // namespace npfem
