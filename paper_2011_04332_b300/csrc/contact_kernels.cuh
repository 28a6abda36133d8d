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
//   k_scatter  vertices into bucket order, with their position relative to their grid
//              cell (float) and their cell index
//   k_query    per vertex: the 27 neighbouring grid cells; a float pre-filter on the
//              cell-relative positions, then the exact FP64 squared distance, evaluated
//              as (dx*dx + dy*dy) + dz*dz without contraction so that every decision is
//              the one an FP64 evaluation in that order takes
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
  float4* sortpos;           // [N] cell-relative position + cell id, bucket order
  double* nrm;               // [N][3] unit vertex normals
  int32_t* ccount;           // [N] matches per vertex (0..2)
  int32_t* cvertex;          // [N][2] matched vertex (-1: unused)
  double* cplane;            // [N][2][4] normal, offset n . (x_j - x_anchor(cell of i))
};

__device__ __forceinline__ int grid_coord(double v, double h_inv) { return (int)floor(v * h_inv); }

__device__ __forceinline__ uint32_t grid_hash(int ix, int iy, int iz, uint32_t mask) {
  return (((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^ ((uint32_t)iz * 83492791u)) & mask;
}

// Unit area-weighted vertex normals of the cells of one type (one warp per cell).  The
// incidence list of a vertex holds its triangle corners in triangle order, so the sum
// runs over the incident triangles in that order.
template <typename S>
__global__ void __launch_bounds__(128) npfem_k_normals(DevTypeView<S> ty, const int32_t* cells, int ncells,
                                                       const int64_t* offsets, int64_t Nt, const S* x, double* nrm) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int c = warp; c < ncells; c += nwarps) {
    const int64_t off = offsets[cells[c]];
    for (int v = lane; v < ty.n; v += 32) {
      double sx = 0.0, sy = 0.0, sz = 0.0;
      const int e0 = __ldg(&ty.inc_ptr[v]), e1 = __ldg(&ty.inc_ptr[v + 1]);
      for (int e = e0; e < e1; ++e) {
        const int code = __ldg(&ty.inc_code[e]);
        if (code < 0) continue;
        const int t = code / 3;
        const int64_t i0 = off + __ldg(&ty.tris[3 * t]), i1 = off + __ldg(&ty.tris[3 * t + 1]),
                      i2 = off + __ldg(&ty.tris[3 * t + 2]);
        const double ax = (double)x[i1] - (double)x[i0], ay = (double)x[Nt + i1] - (double)x[Nt + i0],
                     az = (double)x[2 * Nt + i1] - (double)x[2 * Nt + i0];
        const double bx = (double)x[i2] - (double)x[i0], by = (double)x[Nt + i2] - (double)x[Nt + i0],
                     bz = (double)x[2 * Nt + i2] - (double)x[2 * Nt + i0];
        sx += ay * bz - az * by;
        sy += az * bx - ax * bz;
        sz += ax * by - ay * bx;
      }
      const double inv = 1.0 / sqrt(sx * sx + sy * sy + sz * sz);
      double* o = nrm + 3 * (off + v);
      o[0] = sx * inv;
      o[1] = sy * inv;
      o[2] = sz * inv;
    }
  }
}

template <typename S>
__global__ void npfem_k_hash(ContactParams C, const S* x) {
  const int64_t Nt = C.n_total;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nt; i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = grid_coord((double)x[i], C.h_inv), iy = grid_coord((double)x[Nt + i], C.h_inv),
              iz = grid_coord((double)x[2 * Nt + i], C.h_inv);
    const uint32_t k = grid_hash(ix, iy, iz, C.mask);
    C.key[i] = (int32_t)k;
    atomicAdd(&C.count[k], 1);
  }
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
    const double px = (double)x[i], py = (double)x[Nt + i], pz = (double)x[2 * Nt + i];
    const int ix = grid_coord(px, C.h_inv), iy = grid_coord(py, C.h_inv), iz = grid_coord(pz, C.h_inv);
    const int pos = atomicAdd(&C.cursor[C.key[i]], 1);
    C.sorted[pos] = (int32_t)i;
    C.sortpos[pos] = make_float4((float)(px - ix * C.h), (float)(py - iy * C.h), (float)(pz - iz * C.h),
                                 __int_as_float(C.vcell[i]));
  }
}

struct Match {
  double d2;
  int b, j;
};

// (d2, b) order across cells; within one cell the nearer vertex, then the smaller index.
__device__ __forceinline__ bool match_before(double d2, int b, const Match& m) {
  return d2 < m.d2 || (d2 == m.d2 && b < m.b);
}

__device__ __forceinline__ void offer(Match* s, double d2, int b, int j) {
  if (b == s[0].b || b == s[1].b) {
    const int k = b == s[0].b ? 0 : 1;
    if (d2 < s[k].d2 || (d2 == s[k].d2 && j < s[k].j)) {
      s[k].d2 = d2;
      s[k].j = j;
    }
  } else if (match_before(d2, b, s[1])) {
    s[1] = Match{d2, b, j};
  }
  if (match_before(s[1].d2, s[1].b, s[0])) {
    const Match t = s[0];
    s[0] = s[1];
    s[1] = t;
  }
}

template <typename S>
__global__ void __launch_bounds__(128) npfem_k_query(ContactParams C, const S* x) {
  const int64_t Nt = C.n_total;
  // float pre-filter: cell-relative positions carry at most a few 2^-24 h of error, so
  // a margin of 1e-4 r^2 never rejects a vertex that is inside the radius
  const float r2f = (float)(C.r2 * (1.0 + 1e-4));
  const float hf = (float)C.h;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < Nt; i += (int64_t)gridDim.x * blockDim.x) {
    const int a = C.vcell[i];
    const double px = (double)x[i], py = (double)x[Nt + i], pz = (double)x[2 * Nt + i];
    const int ix = grid_coord(px, C.h_inv), iy = grid_coord(py, C.h_inv), iz = grid_coord(pz, C.h_inv);
    const float rx = (float)(px - ix * C.h), ry = (float)(py - iy * C.h), rz = (float)(pz - iz * C.h);
    Match s[kContactSlots] = {{1e300, 0x7fffffff, -1}, {1e300, 0x7fffffff, -1}};
    for (int oz = -1; oz <= 1; ++oz)
      for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
          const uint32_t k = grid_hash(ix + ox, iy + oy, iz + oz, C.mask);
          const int q1 = C.start[k + 1];
          for (int q = C.start[k]; q < q1; ++q) {
            const float4 sp = C.sortpos[q];
            const int b = __float_as_int(sp.w);
            if (b == a) continue;
            const float fx = (sp.x + (float)ox * hf) - rx, fy = (sp.y + (float)oy * hf) - ry,
                        fz = (sp.z + (float)oz * hf) - rz;
            if (fx * fx + fy * fy + fz * fz > r2f) continue;
            const int j = C.sorted[q];
            const double dx = px - (double)x[j], dy = py - (double)x[Nt + j], dz = pz - (double)x[2 * Nt + j];
            const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            if (!(d2 < C.r2)) continue;
            offer(s, d2, b, j);
          }
        }
    const int64_t anc = C.offsets[a];
    const double axx = (double)x[anc], ayy = (double)x[Nt + anc], azz = (double)x[2 * Nt + anc];
    int cnt = 0;
#pragma unroll
    for (int m = 0; m < kContactSlots; ++m) {
      double* pl = C.cplane + 8 * i + 4 * m;
      if (s[m].j >= 0) {
        const int j = s[m].j;
        const double nx = C.nrm[3 * j], ny = C.nrm[3 * j + 1], nz = C.nrm[3 * j + 2];
        pl[0] = nx;
        pl[1] = ny;
        pl[2] = nz;
        pl[3] = nx * ((double)x[j] - axx) + ny * ((double)x[Nt + j] - ayy) + nz * ((double)x[2 * Nt + j] - azz);
        C.cvertex[2 * i + m] = j;
        cnt = m + 1;
      } else {
        pl[0] = pl[1] = pl[2] = pl[3] = 0.0;
        C.cvertex[2 * i + m] = -1;
      }
    }
    C.ccount[i] = cnt;
  }
}

}  // namespace npfem
