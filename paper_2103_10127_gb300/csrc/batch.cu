// Batched RAV multigrid: many independent problems of uneven size, each with
// nrhs right-hand sides, advanced together.
//
// * Vectors of a batch are RHS-interleaved: entry (row, k) at row * nrhs + k,
//   so every matrix, transfer or inverse entry loaded from HBM serves all
//   right-hand sides.
// * Each phase of the V-cycle (residual, subdomain apply, restriction, coarse
//   solve, prolongation) is one kernel launch over every (problem, level) that
//   takes part in it at that depth below the finest grid; blocks find their
//   problem by binary search in a block-offset table.  Problems whose
//   hierarchy is shallower reach their coarse solve at a smaller depth.
// * The per-(problem, level) descriptors live in device memory, so the whole
//   batched cycle is captured once into a CUDA graph and replayed, the
//   callers' vector pointers being updated in the descriptors between replays.
// * Per right-hand side the kernels add in the same order as the one-problem
//   kernels, so a batched cycle reproduces the single-problem cycle bit for bit.
// * Launch shapes (threads per block of the residual and apply kernels) are
//   chosen at set-up by timing the candidates on the batch's finest levels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cmath>
#include <type_traits>
#include <vector>

#include "box.cuh"
#include "common.cuh"
#include "cpasync.cuh"
#include "tcgen05.cuh"

namespace rav {

struct BLevel {
  Geo g;
  Geo gc;  // next coarser level (restriction target, prolongation source)
  int64_t nslice;
  const int32_t* sperm;
  const int64_t* sptr;
  const int32_t* slen;
  const int32_t* scol;
  const double* sval;
  const void* inv;  // dense owned rows of the RAV inverses (float or double)
  const double* omega;
  int64_t units;
  XferTab tab;      // interpolation into this level from the coarser one
  double* x;        // n x nrhs
  double* b;
  double* r;
  double* xc;       // coarser level's x and b
  double* bc;
  float* r32;       // fp32 batches: r rounded to fp32 (the apply's input), else null
  float* bc32;      // coarser level's r32: its b rounded, written by the restriction
  const double* cinv;  // bordered coarse inverse (coarsest level only)
  int problem;
  // 2-D Q2-Q1, fp32 rows, 8 RHS: the owned rows shared by every interior
  // subdomain of this level (vertices 2 .. N-2 per axis), split into tf32 high
  // and low parts in the tensor-core operand layout (2 x 4096 bytes), or null
  // when the level's interior subdomains do not share them
  const float* gtc;
  // fp32 residual on depths below the finest (batch_set_coarse_residual_f32):
  // the operator values in fp32 (slot order of sval) and a work copy of x in
  // fp32 (n x nrhs); null where the level keeps the fp64 residual
  const float* sval32;
  float* x32;
  // fp32 transfers (batch_set_transfers_f32): the weights of tab in fp32 and
  // the fp32 copy of the coarser level's x prolongated into this level
  XferTabT<float> tab32;
  float* xc32;
};

__device__ __forceinline__ int find_entry(const int64_t* __restrict__ first, int ne, int64_t blk) {
  int lo = 0, hi = ne;  // first[lo] <= blk < first[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (first[mid] <= blk) lo = mid;
    else hi = mid;
  }
  return lo;
}

// NR consecutive residual values of one row (RHS-interleaved, so the row's
// values are contiguous and 4*NR- or 8*NR-byte aligned) in as few loads as the
// alignment allows.
template <typename A, int NR>
__device__ __forceinline__ void load_row(const A* __restrict__ p, A* out) {
  if constexpr (std::is_same<A, float>::value && NR % 4 == 0) {
#pragma unroll
    for (int j = 0; j < NR; j += 4) {
      const float4 v = *reinterpret_cast<const float4*>(p + j);
      out[j] = v.x;
      out[j + 1] = v.y;
      out[j + 2] = v.z;
      out[j + 3] = v.w;
    }
  } else if constexpr (NR % 2 == 0) {
    using V2 = typename std::conditional<std::is_same<A, float>::value, float2, double2>::type;
#pragma unroll
    for (int j = 0; j < NR; j += 2) {
      const V2 v = *reinterpret_cast<const V2*>(p + j);
      out[j] = v.x;
      out[j + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < NR; ++j) out[j] = p[j];
  }
}

// x of every row of each entry rounded to fp32 (the residual phase's block
// layout: one thread per row slot, and every row has a slot).
template <int NR>
__global__ void kb_x_to_f32(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne) {
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const int64_t t = (blockIdx.x - first[e]) * (int64_t)blockDim.x + threadIdx.x;
  if (t >= lv.g.n) return;
#pragma unroll
  for (int j = 0; j < NR; ++j) lv.x32[t * NR + j] = (float)lv.x[t * NR + j];
}

// The operator values of one level rounded to fp32 (set-up).
__global__ void kb_vals_to_f32(const double* __restrict__ v, int64_t n, float* __restrict__ v32) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v32[i] = (float)v[i];
}

// r = b - L x for every right-hand side (same addition order per RHS as
// k_residual_sell), with per-block partial sums of r^2 per RHS when part != 0.
template <int NR>
__global__ void kb_residual(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne,
                            double* __restrict__ part) {
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const int64_t t = (blockIdx.x - first[e]) * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nslots = lv.nslice * 32;
  double sq[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) sq[j] = 0.0;
  if (t < nslots) {
    const int64_t s = t >> 5;
    const int32_t row = lv.sperm[t];
    const int len = lv.slen[s];
    const int64_t base = lv.sptr[s] + (t & 31);
    double a0[NR], a1[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) a0[j] = a1[j] = 0.0;
    if (len > 1) {
      const int32_t* c = lv.scol + base;
      const double* v = lv.sval + base;
      const int full = len & ~7;
      for (int k = 0; k < full; k += 2) {
        const double v0 = ld_stream(v + 32 * k), v1 = ld_stream(v + 32 * (k + 1));
        double x0[NR], x1[NR];
        load_row<double, NR>(lv.x + (int64_t)ld_stream(c + 32 * k) * NR, x0);
        load_row<double, NR>(lv.x + (int64_t)ld_stream(c + 32 * (k + 1)) * NR, x1);
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          a0[j] += v0 * x0[j];
          a1[j] += v1 * x1[j];
        }
      }
      for (int k = full; k < len; ++k) {
        const double v0 = ld_stream(v + 32 * k);
        double x0[NR];
        load_row<double, NR>(lv.x + (int64_t)ld_stream(c + 32 * k) * NR, x0);
#pragma unroll
        for (int j = 0; j < NR; ++j) a0[j] += v0 * x0[j];
      }
    }
    if (row >= 0) {
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const double rv = len > 1 ? lv.b[(int64_t)row * NR + j] - (a0[j] + a1[j]) : 0.0;
        lv.r[(int64_t)row * NR + j] = rv;
        if (lv.r32) lv.r32[(int64_t)row * NR + j] = (float)rv;
        sq[j] = rv * rv;
      }
    }
  }
  if (part) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const double bs = block_sum(sq[j]);
      if (threadIdx.x == 0) part[blockIdx.x * NR + j] = bs;
    }
  }
}

// The same residual on a depth below the finest with fp32 operator values and
// x (batch_set_coarse_residual_f32): products summed in fp32 in the same
// order, r = b - sum formed in fp64.
template <int NR>
__global__ void kb_residual_f32(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne) {
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const int64_t t = (blockIdx.x - first[e]) * (int64_t)blockDim.x + threadIdx.x;
  if (t >= lv.nslice * 32) return;
  const int64_t s = t >> 5;
  const int32_t row = lv.sperm[t];
  const int len = lv.slen[s];
  const int64_t base = lv.sptr[s] + (t & 31);
  float a0[NR], a1[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) a0[j] = a1[j] = 0.f;
  if (len > 1) {
    const int32_t* c = lv.scol + base;
    const float* v = lv.sval32 + base;
    const int full = len & ~7;
    for (int k = 0; k < full; k += 2) {
      const float v0 = ld_stream(v + 32 * k), v1 = ld_stream(v + 32 * (k + 1));
      float x0[NR], x1[NR];
      load_row<float, NR>(lv.x32 + (int64_t)ld_stream(c + 32 * k) * NR, x0);
      load_row<float, NR>(lv.x32 + (int64_t)ld_stream(c + 32 * (k + 1)) * NR, x1);
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        a0[j] += v0 * x0[j];
        a1[j] += v1 * x1[j];
      }
    }
    for (int k = full; k < len; ++k) {
      const float v0 = ld_stream(v + 32 * k);
      float x0[NR];
      load_row<float, NR>(lv.x32 + (int64_t)ld_stream(c + 32 * k) * NR, x0);
#pragma unroll
      for (int j = 0; j < NR; ++j) a0[j] += v0 * x0[j];
    }
  }
  if (row >= 0) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const double rv = len > 1 ? lv.b[(int64_t)row * NR + j] - (double)(a0[j] + a1[j]) : 0.0;
      lv.r[(int64_t)row * NR + j] = rv;
      if (lv.r32) lv.r32[(int64_t)row * NR + j] = (float)rv;
    }
  }
}

// Sum of the partials of each (problem, RHS): norms[p * NR + j] = sqrt(sum).
template <int NR>
__global__ void kb_norm_final(const int64_t* __restrict__ first, const int* __restrict__ prob, int ne,
                              const double* __restrict__ part, double* __restrict__ norms) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne * NR) return;
  const int e = t / NR, j = t % NR;
  double s = 0.0;
  for (int64_t blk = first[e]; blk < first[e + 1]; ++blk) s += part[blk * NR + j];
  norms[prob[e] * NR + j] = sqrt(s);
}

// RAV apply with dense owned rows, all right-hand sides at once (same order
// per RHS as k_rav_apply).  use_b: the residual is b (x entered as 0).
template <int D, typename T, int NR>
__global__ void kb_apply(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne, int use_b) {
  using B = BoxT<D>;
  constexpr int NC = B::NC, RB = B::RB, NCH = B::NCH;
  using Acc = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const int64_t u = (blockIdx.x - first[e]) * (int64_t)blockDim.x + threadIdx.x;
  if (u >= lv.units) return;
  const Geo& g = lv.g;
  // fp32 storage reads the fp32-rounded residual (r32 holds b itself after the
  // restriction, when x entered as 0)
  const Acc* __restrict__ r =
      std::is_same<T, double>::value ? (const Acc*)(use_b ? lv.b : lv.r) : (const Acc*)lv.r32;
  const int64_t p = u / NCH;
  const int h = (int)(u % NCH);
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  // interior subdomains of a level with shared rows go through kb_apply_tc
  if (D == 2 && lv.gtc && v[0] >= 2 && v[0] <= g.N - 2 && v[1] >= 2 && v[1] <= g.N - 2) return;
  const int M = (int)g.M;
  int alo[3] = {0, 0, 0}, ahi[3] = {0, 0, 0};
#pragma unroll
  for (int d = 0; d < D; ++d) {
    alo[d] = 2 - 2 * v[d] > 0 ? 2 - 2 * v[d] : 0;
    ahi[d] = 2 * g.N - 2 * v[d] + 2 < 4 ? 2 * g.N - 2 * v[d] + 2 : 4;
  }
  int64_t base = 0;
#pragma unroll
  for (int d = D - 1; d >= 0; --d) base = base * M + (2 * v[d] - 2);
  base *= D;
  const T* ip = static_cast<const T*>(lv.inv) + ((u >> 5) * NC * RB) * 32 + (u & 31);
  Acc acc[RB][NR];
#pragma unroll
  for (int i = 0; i < RB; ++i)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[i][j] = 0;
  int k = 0;
  for (int a2 = 0; a2 < (D == 3 ? 5 : 1); ++a2) {
    const bool v2 = D == 2 || (a2 >= alo[2] && a2 <= ahi[2]);
    for (int a1 = 0; a1 < 5; ++a1) {
      const bool v1 = v2 && a1 >= alo[1] && a1 <= ahi[1];
      const int64_t rowoff = base + (int64_t)D * M * (a1 + (int64_t)M * a2);
      for (int a0 = 0; a0 < 5; ++a0) {
        const bool vv = v1 && a0 >= alo[0] && a0 <= ahi[0];
        for (int c = 0; c < D; ++c) {
          Acc ra[NR];
          if (vv) {
            load_row<Acc, NR>(r + (rowoff + D * a0 + c) * NR, ra);
          } else {
#pragma unroll
            for (int j = 0; j < NR; ++j) ra[j] = 0;
          }
#pragma unroll
          for (int i = 0; i < RB; ++i) {
            const Acc q = (Acc)ip[(k * RB + i) * 32];
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[i][j] += q * ra[j];
          }
          ++k;
        }
      }
    }
  }
  {
    Acc ra[NR];
    load_row<Acc, NR>(r + (g.n_u + p) * NR, ra);
#pragma unroll
    for (int i = 0; i < RB; ++i) {
      const Acc q = (Acc)ip[(k * RB + i) * 32];
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[i][j] += q * ra[j];
    }
  }
  const double om = lv.omega[p];
#pragma unroll
  for (int i = 0; i < RB; ++i) {
    const int jrow = h * RB + i;
    int64_t dof = -1;
    if (jrow < B::NR - 1) {
      const int q = jrow / D, c = jrow % D;
      int64_t J[3] = {0, 0, 0};
      bool ok = true;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        J[d] = 2 * v[d] + ((q >> d) & 1);
        ok &= (J[d] >= 1) & (J[d] <= 2 * g.N - 1);
      }
      if (ok) dof = D * node_id_t<D>(g, J) + c;
    } else {
      dof = g.n_u + p;
    }
    if (dof >= 0) {
#pragma unroll
      for (int j = 0; j < NR; ++j) lv.x[dof * NR + j] += om * (double)acc[i][j];
    }
  }
}

// ---- tiled apply: 2-D Q2-Q1, fp32 rows, 8 right-hand sides ------------------
// kb_apply's thread per subdomain gathers each box node's 8-wide residual row
// and updates its owned rows of x where the lanes of a warp sit two nodes
// apart: every load or store of a warp touches 32 cache lines, and those L1
// wavefronts, not HBM, set its time.  Here a block takes 32 x TY vertices (a
// warp spans one row of 32 vertices, so the interleaved stored rows stay one
// warp-wide load; SPLIT warps per row share its owned rows).  The fp32 residual of the block's boxes, (2*32+3) x (2*TY+3) nodes x
// 2 components x 8 RHS, is copied once into shared memory by coalesced 16-byte
// cp.async (zero outside the grid, where kb_apply reads zero); each thread
// forms kb_apply's sums in kb_apply's order from there; the velocity
// corrections go back through the same buffer and are added to x by rows of
// owned nodes (contiguous 16-byte pieces), the pressure correction directly.
// Results equal kb_apply's bit for bit.
constexpr int kTileX = 32;  // vertices per block row (the lanes of a warp)

// Byte offset of 16-byte chunk q (0..3: component q/2, RHS 4(q%2)..4(q%2)+3)
// of node ln in a tile buffer: two 64-byte nodes per 128-byte line, the chunk
// slot XOR-ed with the line index, so that the 8 lanes of a quarter-warp
// (consecutive vertices: nodes two apart, consecutive lines) take 8 distinct
// slots, i.e. all 32 banks.
__device__ __forceinline__ int tile_off(int ln, int q) {
  const int line = ln >> 1;
  return line * 128 + (((((ln & 1) << 2) | q) ^ (line & 7)) << 4);
}
template <int TY>
struct TileShape {
  static constexpr int SX = 2 * kTileX + 3, SY = 2 * TY + 3;  // staged box nodes per axis
  static constexpr int OX = 2 * kTileX, OY = 2 * TY;          // owned nodes per axis
  static constexpr int BYTES = (SX * SY + 1) / 2 * 128;       // >= OX * OY / 2 * 128
};

// Sums of owned rows I0 .. I1-1 of the subdomain at (tx, ty) of the block
// (kb_apply's order: box positions k = 2 (a0 + 5 a1) + c, pressure last).
template <int I0, int I1, int RMAX>
__device__ __forceinline__ void tile_rows(const unsigned char* sm, int sx, const float* __restrict__ ip,
                                          const float* __restrict__ rp, int tx, int ty, float (&acc)[RMAX][8]) {
  constexpr int RB = BoxT<2>::RB;
  int k = 0;
  for (int a1 = 0; a1 < 5; ++a1) {
    for (int a0 = 0; a0 < 5; ++a0) {
      const int ln = (2 * ty + a1) * sx + 2 * tx + a0;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float4 lo = *reinterpret_cast<const float4*>(sm + tile_off(ln, 2 * c));
        const float4 hi = *reinterpret_cast<const float4*>(sm + tile_off(ln, 2 * c + 1));
        const float ra[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
        for (int i = I0; i < I1; ++i) {
          const float q = ip[(k * RB + i) * 32];
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i - I0][j] += q * ra[j];
        }
        ++k;
      }
    }
  }
  float ra[8];
  load_row<float, 8>(rp, ra);
#pragma unroll
  for (int i = I0; i < I1; ++i) {
    const float q = ip[(k * RB + i) * 32];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i - I0][j] += q * ra[j];
  }
}

// Owned rows I0 .. I1-1 out: row i < 8 (node 2v + (q & 1, q >> 1), q = i / 2,
// component i % 2) into the block's correction buffer, row 8 (the pressure)
// straight into x.
template <int I0, int I1, int RMAX>
__device__ __forceinline__ void tile_store(unsigned char* sm, int ox, int tx, int ty, double om,
                                           double* __restrict__ xp, const float (&acc)[RMAX][8]) {
#pragma unroll
  for (int i = I0; i < I1; ++i) {
    if (i < 8) {
      const int q = i >> 1, c = i & 1;
      const int on = (2 * ty + (q >> 1)) * ox + 2 * tx + (q & 1);
      const float* a = acc[i - I0];
      *reinterpret_cast<float4*>(sm + tile_off(on, 2 * c)) = make_float4(a[0], a[1], a[2], a[3]);
      *reinterpret_cast<float4*>(sm + tile_off(on, 2 * c + 1)) = make_float4(a[4], a[5], a[6], a[7]);
    } else {
      double2* x2 = reinterpret_cast<double2*>(xp);
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        double2 xv = x2[h];
        xv.x += om * (double)acc[i - I0][2 * h];
        xv.y += om * (double)acc[i - I0][2 * h + 1];
        x2[h] = xv;
      }
    }
  }
}

// SPLIT = 1: one thread per subdomain, all 9 owned rows (72 accumulators).
// SPLIT = 2: two warps per row of vertices, rows 0-3 and rows 4-8 of the same
// subdomains (at most 40 accumulators, twice the warps per SM); each reads the
// whole staged box and its own rows of the stored inverse.
template <int TY, int SPLIT>
__global__ void __launch_bounds__(kTileX * TY * SPLIT, SPLIT == 1 ? 16 / TY : (TY == 2 ? 5 : 2))
    kb_apply_tile(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne) {
  using B = BoxT<2>;
  using S = TileShape<TY>;
  constexpr int NC = B::NC, RB = B::RB, NR = 8, NT = kTileX * TY * SPLIT;
  constexpr int RMAX = SPLIT == 1 ? RB : 5, IH = SPLIT == 1 ? RB : 4;  // rows of the first warp: 0 .. IH-1
  static_assert(B::NCH == 1 && RB == 9, "one thread per subdomain, 9 owned rows");
  __shared__ __align__(128) unsigned char sm[S::BYTES];
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const Geo& g = lv.g;
  const int N = g.N, V = N + 1, M = 2 * N + 1;
  const int ntx = (V + kTileX - 1) / kTileX;
  const int lb = (int)(blockIdx.x - first[e]);
  const int vx0 = (lb % ntx) * kTileX, vy0 = (lb / ntx) * TY;
  const int w = threadIdx.x >> 5, tx = threadIdx.x & 31, ty = w / SPLIT, h = w % SPLIT;
  const float* __restrict__ r = lv.r32;
  // 1. the residual of the block's boxes: nodes 2*v0 - 2 + (0 .. S-1) per axis
  const int gx0 = 2 * vx0 - 2, gy0 = 2 * vy0 - 2;
  for (int idx = threadIdx.x; idx < S::SX * S::SY * 4; idx += NT) {
    const int ln = idx >> 2, q = idx & 3;
    const int gx = gx0 + ln % S::SX, gy = gy0 + ln / S::SX;
    const bool ok = gx >= 0 && gx < M && gy >= 0 && gy < M;
    st_copy16z(sm + tile_off(ln, q), ok ? r + ((int64_t)gy * M + gx) * 16 + 4 * q : r, ok);
  }
  st_commit();
  st_wait<0>();
  __syncthreads();
  // 2. kb_apply's sums (tensor-core levels leave their interior subdomains to kb_apply_tc)
  const int vx = vx0 + tx, vy = vy0 + ty;
  const bool run = vx <= N && vy <= N && !(lv.gtc && vx >= 2 && vx <= N - 2 && vy >= 2 && vy <= N - 2);
  const int64_t p = (int64_t)vy * V + vx;
  float acc[RMAX][NR];
#pragma unroll
  for (int i = 0; i < RMAX; ++i)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[i][j] = 0.f;
  const float* ip = static_cast<const float*>(lv.inv) + ((p >> 5) * NC * RB) * 32 + (p & 31);
  const float* rp = r + (g.n_u + p) * NR;
  if (run) {
    if (h == 0) tile_rows<0, IH, RMAX>(sm, S::SX, ip, rp, tx, ty, acc);
    else tile_rows<4, RB, RMAX>(sm, S::SX, ip, rp, tx, ty, acc);
  }
  __syncthreads();  // the staged residual is no longer read
  if (run) {
    const double om = lv.omega[p];
    double* xp = lv.x + (g.n_u + p) * NR;
    if (h == 0) tile_store<0, IH, RMAX>(sm, S::OX, tx, ty, om, xp, acc);
    else tile_store<4, RB, RMAX>(sm, S::OX, tx, ty, om, xp, acc);
  }
  __syncthreads();
  // x of the owned nodes, 16 bytes (two RHS of one component) per step: node
  // J = 2 v0 + (on % OX, on / OX), pair w -> component w / 4, RHS 2(w % 4), +1;
  // interior nodes only, owner vertex J / 2 (skipped where kb_apply_tc owns it)
  for (int idx = threadIdx.x; idx < S::OX * S::OY * 8; idx += NT) {
    const int on = idx >> 3, pw = idx & 7;
    const int Jx = 2 * vx0 + on % S::OX, Jy = 2 * vy0 + on / S::OX;
    if (Jx < 1 || Jx > 2 * N - 1 || Jy < 1 || Jy > 2 * N - 1) continue;
    const int ox = Jx >> 1, oy = Jy >> 1;
    if (lv.gtc && ox >= 2 && ox <= N - 2 && oy >= 2 && oy <= N - 2) continue;
    const double om = lv.omega[(int64_t)oy * V + ox];
    const float2 a = *reinterpret_cast<const float2*>(sm + tile_off(on, pw >> 1) + 8 * (pw & 1));
    double2* xq = reinterpret_cast<double2*>(lv.x + ((int64_t)Jy * M + Jx) * 16) + pw;
    double2 xv = *xq;
    xv.x += om * (double)a.x;
    xv.y += om * (double)a.y;
    *xq = xv;
  }
}

// ---- shared-inverse apply on the tensor cores ----------------------------------
// On a uniform grid with constant viscosity every interior subdomain of a level
// (vertices 2 .. N-2 per axis: the whole 5 x 5 node box free) has the same local
// system L_i, so the same owned rows G = (L_i^{-1})_{owned,:} (9 x 51 in 2-D,
// Eq. 13 with the restricted rows of Sec. 4.3).  For 16 such subdomains and the
// 8 right-hand sides of each, the restricted local solves are one small GEMM
//   Y[(16 x 8) x 9] = Rloc[(16 x 8) x 51] G^T,
// rows = (subdomain, right-hand side), Rloc row = the gathered residual box
// (Sec. 3's restriction R_i).  It runs as tcgen05.mma kind::tf32, M = 128,
// N = 16 (9 used), K = 64 (51 used), fp32 accumulation in tensor memory, in
// three passes hi*hi + hi*lo + lo*hi of operands split into tf32 parts
// (x = hi + lo, hi = x with the low 13 mantissa bits cleared), which keeps
// each product's relative error near 2^-20 instead of tf32's 2^-11.
// Per tile: the 256 threads of a block store Rloc, gathered from the fp32
// residual into registers while the previous tile's MMAs ran, into shared
// memory (core matrices of 8 rows x 16 bytes, K-major, no swizzle; one row
// group = one subdomain's 8 right-hand sides; a 16-byte pad between groups
// spreads the stores over all banks), one thread issues the 24 MMAs and
// commits them to an mbarrier, the threads load the next tile's rows, then
// read the 128 x 16 accumulator from tensor memory (two warps per lane
// quarter, five owned rows each) and add omega_i y to the owned DoFs of x
// (restricted scatter, disjoint per subdomain, no atomics).  Waits on the
// mbarrier are bounded: a wait that gives up sets *err and the block stops
// after a second bounded wait for its MMAs, freeing its tensor memory.
// Boundary subdomains of the same level stay on kb_apply.
constexpr int kTcP = 16;                       // subdomains per tile (x 8 RHS = M = 128)
constexpr int kTcSboA = 16 * 128 + 16;         // bytes between row groups of Rloc
constexpr int kTcABytes = kTcP * kTcSboA;      // 33,024
constexpr int kTcBBytes = 2 * 16 * 128;        // 16 x 64 tf32, row groups 2048 bytes apart
constexpr int kTcSmem = 2 * kTcABytes + 2 * kTcBBytes + 16;
constexpr long kTcWaitProbes = 1L << 22;

__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xffffe000u); }

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
  for (long i = 0; i < kTcWaitProbes; ++i)
    if (tc::mbar_try_wait(bar, parity)) return true;
  return false;
}

// Residual rows of one tile gathered into registers: thread task i (of 4)
// covers subdomain pl = 8 (w & 1) + lane / 4 and box position
// kk = 4 (w / 2) + lane % 4, w = warp + 8 i; 8 right-hand sides each.
struct TcGather {
  float4 v[4][2];
};
__device__ __forceinline__ void tc_gather_load(const BLevel& lv, int64_t t0, int warp, int lane, TcGather& gr) {
  const Geo& g = lv.g;
  const int ni = g.N - 3;
  const int64_t nint = (int64_t)ni * ni;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int w = warp + 8 * i;
    const int pl = 8 * (w & 1) + (lane >> 2);
    const int kk = 4 * (w >> 1) + (lane & 3);
    const int64_t idx = t0 + pl;
    gr.v[i][0] = gr.v[i][1] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (idx < nint && kk <= 50) {
      const int vx = 2 + (int)(idx % ni), vy = 2 + (int)(idx / ni);
      int64_t row;
      if (kk == 50) {
        row = g.n_u + vx + (int64_t)(g.N + 1) * vy;
      } else {
        const int a = kk >> 1;
        row = 2 * ((2 * vx - 2 + a % 5) + g.M * (2 * vy - 2 + a / 5)) + (kk & 1);
      }
      const float4* src = reinterpret_cast<const float4*>(lv.r32 + row * 8);
      gr.v[i][0] = src[0];
      gr.v[i][1] = src[1];
    }
  }
}
__device__ __forceinline__ void tc_gather_store(const TcGather& gr, int warp, int lane, uint8_t* a_hi, uint8_t* a_lo) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int w = warp + 8 * i;
    const int pl = 8 * (w & 1) + (lane >> 2);
    const int kk = 4 * (w >> 1) + (lane & 3);
    const int off = pl * kTcSboA + (kk >> 2) * 128 + (kk & 3) * 4;
    const float v[8] = {gr.v[i][0].x, gr.v[i][0].y, gr.v[i][0].z, gr.v[i][0].w,
                        gr.v[i][1].x, gr.v[i][1].y, gr.v[i][1].z, gr.v[i][1].w};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float hi = tf32_hi(v[j]);
      *reinterpret_cast<float*>(a_hi + off + 16 * j) = hi;
      *reinterpret_cast<float*>(a_lo + off + 16 * j) = v[j] - hi;
    }
  }
}

// 8 warps: all gather; thread 0 issues the MMAs; warps w and w + 4 read the
// same accumulator rows (lane quarter w % 4) and write owned rows 0-4 and 5-8.
// The next tile's residual rows are loaded into registers while the MMAs of
// the current one run.
__global__ void __launch_bounds__(256) kb_apply_tc(const BLevel* __restrict__ L, const int64_t* __restrict__ first,
                                                   int ne, int* __restrict__ err) {
  extern __shared__ __align__(128) uint8_t tsm[];
  uint8_t* a_hi = tsm;
  uint8_t* a_lo = tsm + kTcABytes;
  uint8_t* b_hi = tsm + 2 * kTcABytes;
  uint8_t* b_lo = b_hi + kTcBBytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(b_lo + kTcBBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(tslot, 32);
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::mbar_init_fence();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  // contiguous tile range per block (neighbouring tiles share residual rows in L2)
  const int64_t ntiles = first[ne];
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t_begin = blockIdx.x * per, t_end = t_begin + per < ntiles ? t_begin + per : ntiles;
  const uint32_t idesc = tc::idesc_tf32(128, 16);
  uint32_t phase = 0;
  int cur = -1;
  bool failed = false;
  TcGather gr;
  int e = t_begin < t_end ? find_entry(first, ne, t_begin) : 0;
  if (t_begin < t_end) tc_gather_load(L[e], (t_begin - first[e]) * kTcP, warp, lane, gr);
  for (int64_t tile = t_begin; tile < t_end; ++tile) {
    const BLevel& lv = L[e];
    const Geo& g = lv.g;
    if (e != cur) {  // this level's shared rows, both tf32 parts
      const uint4* src = reinterpret_cast<const uint4*>(lv.gtc);
      uint4* dst = reinterpret_cast<uint4*>(b_hi);
      for (int i = tid; i < 2 * kTcBBytes / 16; i += 256) dst[i] = src[i];
      cur = e;
    }
    const int ni = g.N - 3;  // interior vertices per axis
    const int64_t nint = (int64_t)ni * ni;
    const int64_t t0 = (tile - first[e]) * kTcP;
    tc_gather_store(gr, warp, lane, a_hi, a_lo);
    tc::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t ah = tc::smem_addr(a_hi), al = tc::smem_addr(a_lo);
      const uint32_t bh = tc::smem_addr(b_hi), bl = tc::smem_addr(b_lo);
#pragma unroll
      for (int k = 0; k < 8; ++k) {  // K = 8 tf32 per MMA: two 16-byte core-matrix columns
        const uint64_t dah = tc::smem_desc(ah + 256 * k, 128, kTcSboA);
        const uint64_t dal = tc::smem_desc(al + 256 * k, 128, kTcSboA);
        const uint64_t dbh = tc::smem_desc(bh + 256 * k, 128, 2048);
        const uint64_t dbl = tc::smem_desc(bl + 256 * k, 128, 2048);
        tc::mma_tf32(tmem, dah, dbh, idesc, k > 0 ? 1u : 0u);
        tc::mma_tf32(tmem, dah, dbl, idesc, 1u);
        tc::mma_tf32(tmem, dal, dbh, idesc, 1u);
      }
      tc::mma_commit(bar);
    }
    // the next tile's residual rows, while the tensor cores work
    const int e_next = tile + 1 < t_end ? find_entry(first, ne, tile + 1) : e;
    if (tile + 1 < t_end) tc_gather_load(L[e_next], (tile + 1 - first[e_next]) * kTcP, warp, lane, gr);
    const bool done = tc_wait(bar, phase);
    failed = __syncthreads_or(!done) != 0;
    if (failed) break;
    phase ^= 1u;
    tc::fence_after_sync();
    float y[16];
    tc::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16), y);
    const int m = (warp & 3) * 32 + lane;  // accumulator row: subdomain m / 8, right-hand side m % 8
    const int64_t idx = t0 + (m >> 3);
    const int rhs = m & 7;
    if (idx < nint) {
      const int vx = 2 + (int)(idx % ni), vy = 2 + (int)(idx / ni);
      const int64_t p = vx + (int64_t)(g.N + 1) * vy;
      const double om = lv.omega[p];
      const int j0 = warp < 4 ? 0 : 5, j1 = warp < 4 ? 5 : 9;
      double* xp[5];
      double xv[5];
#pragma unroll
      for (int jj = 0; jj < 5; ++jj) {  // owned row j: node 2v + (q & 1, q >> 1), q = j / 2, component j % 2
        const int j = j0 + jj;
        xp[jj] = nullptr;
        if (j < j1) {
          const int q = j >> 1;
          const int64_t dof =
              j == 8 ? g.n_u + p : 2 * ((2 * vx + (q & 1)) + g.M * (2 * vy + (q >> 1))) + (j & 1);
          xp[jj] = lv.x + dof * 8 + rhs;
          xv[jj] = *xp[jj];
        }
      }
#pragma unroll
      for (int jj = 0; jj < 5; ++jj)
        if (xp[jj]) *xp[jj] = xv[jj] + om * (double)y[j0 + jj];
    }
    tc::fence_before_sync();
    __syncthreads();
    e = e_next;
  }
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    tc_wait(bar, phase);  // the MMAs of the abandoned tile, bounded again
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 32);
  }
}

// Checks whether every interior subdomain's stored fp32 rows (2-D, one unit
// per subdomain: element (u, j, k) at ((u / 32) NC + k) RB + j) 32 + u % 32)
// equal those of the subdomain at vertex (2, 2) within tol; *bad = 1 if not.
__global__ void kb_shared_check(Geo g, const float* __restrict__ inv, float tol, int* __restrict__ bad) {
  using B = BoxT<2>;
  constexpr int NC = B::NC, RB = B::RB;
  const int ni = g.N - 3;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)ni * ni * RB * NC) return;
  const int64_t idx = e / (RB * NC);
  const int j = (int)((e / NC) % RB), k = (int)(e % NC);
  const int64_t u = (2 + idx % ni) + (int64_t)(g.N + 1) * (2 + idx / ni);
  const int64_t u0 = 2 + (int64_t)(g.N + 1) * 2;
  const float a = inv[((u >> 5) * NC + k) * RB * 32 + j * 32 + (u & 31)];
  const float r = inv[((u0 >> 5) * NC + k) * RB * 32 + j * 32 + (u0 & 31)];
  if (!(fabsf(a - r) <= tol)) atomicExch(bad, 1);
}

// Shared rows of the subdomain at vertex (2, 2) as the B operand: element
// (n, k) (owned row n < 9, box position k < 51; zero elsewhere) of the 16 x 64
// matrix at (n / 8) 2048 + (k / 4) 128 + (n % 8) 16 + (k % 4) 4 bytes, tf32
// high part in the first 4096 bytes, low part in the next.
__global__ void kb_shared_build(Geo g, const float* __restrict__ inv, float* __restrict__ out) {
  using B = BoxT<2>;
  constexpr int NC = B::NC, RB = B::RB;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 16 * 64) return;
  const int n = e / 64, k = e % 64;
  const int64_t u0 = 2 + (int64_t)(g.N + 1) * 2;
  const float v = (n < RB && k < NC) ? inv[((u0 >> 5) * NC + k) * RB * 32 + n * 32 + (u0 & 31)] : 0.f;
  const float hi = tf32_hi(v);
  const int off = ((n >> 3) * 2048 + (k >> 2) * 128 + (n & 7) * 16 + (k & 3) * 4) / 4;
  out[off] = hi;
  out[1024 + off] = v - hi;
}

// Transfer tables and inputs in the transfers' arithmetic type.
template <typename W>
__device__ __forceinline__ const XferTabT<W>& xfer_tab(const BLevel& lv);
template <>
__device__ __forceinline__ const XferTabT<double>& xfer_tab<double>(const BLevel& lv) { return lv.tab; }
template <>
__device__ __forceinline__ const XferTabT<float>& xfer_tab<float>(const BLevel& lv) { return lv.tab32; }
template <typename W>
__device__ __forceinline__ const W* restrict_in(const BLevel& lv);
template <>
__device__ __forceinline__ const double* restrict_in<double>(const BLevel& lv) { return lv.r; }
template <>
__device__ __forceinline__ const float* restrict_in<float>(const BLevel& lv) { return lv.r32; }
template <typename W>
__device__ __forceinline__ const W* prolong_in(const BLevel& lv);
template <>
__device__ __forceinline__ const double* prolong_in<double>(const BLevel& lv) { return lv.xc; }
template <>
__device__ __forceinline__ const float* prolong_in<float>(const BLevel& lv) { return lv.xc32; }

// Restriction into the coarser level (same threads per coarse DoF and the same
// order per RHS as k_restrict_c); also zeroes the coarser iterate.  W = double:
// fp64; W = float (batch_set_transfers_f32): the fp32 residual copy r32, fp32
// weights and sums, bc written in fp64.
template <int D, int NR, typename W>
__global__ void kb_restrict(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne) {
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const Geo &gf = lv.g, &gc = lv.gc;
  const XferTabT<W>& T = xfer_tab<W>(lv);
  const int tl = restrict_split(gc);
  const int64_t gt = (blockIdx.x - first[e]) * (int64_t)blockDim.x + threadIdx.x;
  const int t = (int)(gt / tl), sub = (int)(gt % tl);
  const int Mf = (int)gf.M, Mc = (int)gc.M, nnc = (int)gc.nnode;
  const W* rf = restrict_in<W>(lv);
  W acc[D][NR];
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[c][j] = 0;
  if (t < nnc) {
    int K[3] = {0, 0, 0}, id = t;
    bool bnd = false;
    for (int a = 0; a < D; ++a) {
      K[a] = id % Mc;
      id /= Mc;
      bnd |= (K[a] == 0) | (K[a] == Mc - 1);
    }
    if (!bnd) {
      const int c0 = T.rc2[0][K[0]], c1 = T.rc2[1][K[1]], c2 = D == 3 ? T.rc2[2][K[2]] : 1;
      for (int pr = sub; pr < c2 * c1; pr += tl) {
        const int j2 = pr / c1, j1 = pr % c1;
        const int I2 = D == 3 ? T.rk2[2][7 * K[2] + j2] : 0;
        const W w2 = D == 3 ? T.rw2[2][7 * K[2] + j2] : W(1);
        const int I1 = T.rk2[1][7 * K[1] + j1];
        const W w12 = D == 3 ? w2 * T.rw2[1][7 * K[1] + j1] : T.rw2[1][7 * K[1] + j1];
        const int64_t rowbase = (int64_t)D * Mf * (I1 + (int64_t)Mf * I2);
        for (int j0 = 0; j0 < c0; ++j0) {
          const W ww = w12 * T.rw2[0][7 * K[0] + j0];
          const int64_t bse = rowbase + D * T.rk2[0][7 * K[0] + j0];
#pragma unroll
          for (int c = 0; c < D; ++c)
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[c][j] += ww * rf[(bse + c) * NR + j];
        }
      }
    }
  } else if (t < nnc + (int)gc.n_p) {
    const int Nf1 = gf.N + 1, Nc1 = gc.N + 1;
    int K[3] = {0, 0, 0}, id = t - nnc;
    for (int a = 0; a < D; ++a) { K[a] = id % Nc1; id /= Nc1; }
    const int c0 = T.rc1[0][K[0]], c1 = T.rc1[1][K[1]], c2 = D == 3 ? T.rc1[2][K[2]] : 1;
    for (int pr = sub; pr < c2 * c1; pr += tl) {
      const int j2 = pr / c1, j1 = pr % c1;
      const int V2 = D == 3 ? T.rk1[2][3 * K[2] + j2] : 0;
      const W w2 = D == 3 ? T.rw1[2][3 * K[2] + j2] : W(1);
      const int V1 = T.rk1[1][3 * K[1] + j1];
      const W w12 = D == 3 ? w2 * T.rw1[1][3 * K[1] + j1] : T.rw1[1][3 * K[1] + j1];
      for (int j0 = 0; j0 < c0; ++j0) {
        const W ww = w12 * T.rw1[0][3 * K[0] + j0];
        const int64_t idx = gf.n_u + T.rk1[0][3 * K[0] + j0] + Nf1 * (V1 + (int64_t)Nf1 * V2);
#pragma unroll
        for (int j = 0; j < NR; ++j) acc[0][j] += ww * rf[idx * NR + j];
      }
    }
  }
  for (int o = tl >> 1; o > 0; o >>= 1)
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[c][j] += __shfl_xor_sync(0xffffffffu, acc[c][j], o, tl);
  if (sub != 0) return;
  if (t < nnc) {
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        lv.bc[((int64_t)D * t + c) * NR + j] = (double)acc[c][j];
        if (lv.bc32) lv.bc32[((int64_t)D * t + c) * NR + j] = (float)acc[c][j];
        lv.xc[((int64_t)D * t + c) * NR + j] = 0.0;
      }
  } else if (t < nnc + (int)gc.n_p) {
    const int64_t o = gc.n_u + (t - nnc);
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      lv.bc[o * NR + j] = (double)acc[0][j];
      if (lv.bc32) lv.bc32[o * NR + j] = (float)acc[0][j];
      lv.xc[o * NR + j] = 0.0;
    }
  }
}

// The coarser level's x rounded to fp32 before an fp32 prolongation (the
// prolongation phase's blocks, every coarse row reached by a block-stride loop).
template <int NR>
__global__ void kb_xc_to_f32(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne) {
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const int64_t nt = (first[e + 1] - first[e]) * (int64_t)blockDim.x;
  for (int64_t i = (blockIdx.x - first[e]) * (int64_t)blockDim.x + threadIdx.x; i < lv.gc.n * NR; i += nt)
    lv.xc32[i] = (float)lv.xc[i];
}

// x += P xc (same order per RHS as k_prolong).  W = float: the fp32 copy of xc,
// fp32 weights and sums, added to x in fp64.
template <int D, int NR, typename W>
__global__ void kb_prolong(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne) {
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const Geo &gf = lv.g, &gc = lv.gc;
  const XferTabT<W>& T = xfer_tab<W>(lv);
  const int t = (int)((blockIdx.x - first[e]) * blockDim.x + threadIdx.x);
  const int Mf = (int)gf.M, Mc = (int)gc.M, nnf = (int)gf.nnode;
  const W* xc = prolong_in<W>(lv);
  if (t < nnf) {
    int I[3] = {0, 0, 0}, id = t;
    bool bnd = false;
    for (int a = 0; a < D; ++a) {
      I[a] = id % Mf;
      id /= Mf;
      bnd |= (I[a] == 0) | (I[a] == Mf - 1);
    }
    if (bnd) return;
    const int c0 = T.pc2[0][I[0]], c1 = T.pc2[1][I[1]], c2 = D == 3 ? T.pc2[2][I[2]] : 1;
    W acc[D][NR];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[c][j] = 0;
    for (int j2 = 0; j2 < c2; ++j2) {
      const int K2 = D == 3 ? T.pk2[2][3 * I[2] + j2] : 0;
      const W w2 = D == 3 ? T.pw2[2][3 * I[2] + j2] : W(1);
      for (int j1 = 0; j1 < c1; ++j1) {
        const int K1 = T.pk2[1][3 * I[1] + j1];
        const W w12 = D == 3 ? w2 * T.pw2[1][3 * I[1] + j1] : T.pw2[1][3 * I[1] + j1];
        const int rowbase = D * Mc * (K1 + Mc * K2);
        for (int j0 = 0; j0 < c0; ++j0) {
          const W ww = w12 * T.pw2[0][3 * I[0] + j0];
          const int bse = rowbase + D * T.pk2[0][3 * I[0] + j0];
#pragma unroll
          for (int c = 0; c < D; ++c)
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[c][j] += ww * xc[((int64_t)bse + c) * NR + j];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int j = 0; j < NR; ++j) lv.x[((int64_t)D * t + c) * NR + j] += (double)acc[c][j];
  } else if (t < nnf + (int)gf.n_p) {
    const int Nf1 = gf.N + 1, Nc1 = gc.N + 1;
    int v[3] = {0, 0, 0}, id = t - nnf;
    for (int a = 0; a < D; ++a) { v[a] = id % Nf1; id /= Nf1; }
    const int c0 = T.pc1[0][v[0]], c1 = T.pc1[1][v[1]], c2 = D == 3 ? T.pc1[2][v[2]] : 1;
    W acc[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[j] = 0;
    for (int j2 = 0; j2 < c2; ++j2) {
      const int K2 = D == 3 ? T.pk1[2][2 * v[2] + j2] : 0;
      const W w2 = D == 3 ? T.pw1[2][2 * v[2] + j2] : W(1);
      for (int j1 = 0; j1 < c1; ++j1) {
        const int K1 = T.pk1[1][2 * v[1] + j1];
        const W w12 = D == 3 ? w2 * T.pw1[1][2 * v[1] + j1] : T.pw1[1][2 * v[1] + j1];
        for (int j0 = 0; j0 < c0; ++j0) {
          const W w = w12 * T.pw1[0][2 * v[0] + j0];
          const int64_t idx = gc.n_u + T.pk1[0][2 * v[0] + j0] + Nc1 * (K1 + Nc1 * K2);
#pragma unroll
          for (int j = 0; j < NR; ++j) acc[j] += w * xc[idx * NR + j];
        }
      }
    }
    const int64_t o = gf.n_u + (t - nnf);
#pragma unroll
    for (int j = 0; j < NR; ++j) lv.x[o * NR + j] += (double)acc[j];
  }
}

// ---- stabilised Q1-Q1 (one thread per subdomain / vertex) --------------------
// RAV apply with the dense owned rows of a Q1-Q1 subdomain (structure of
// arrays, element (j, k) of subdomain p at (j NC + k) np + p; same order per
// RHS as k_rav_apply_q1_rows).  use_b: the residual is b (x entered as 0).
template <int D, typename T, int NR>
__global__ void kb_apply_q1(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne, int use_b) {
  constexpr int NV = D == 2 ? 9 : 27, NC = D * NV + 1, NROW = D + 1;
  using Acc = typename std::conditional<std::is_same<T, double>::value, double, float>::type;
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const int64_t p = (blockIdx.x - first[e]) * (int64_t)blockDim.x + threadIdx.x;
  const int64_t np = lv.units;
  if (p >= np) return;
  const Geo& g = lv.g;
  const Acc* __restrict__ r =
      std::is_same<T, double>::value ? (const Acc*)(use_b ? lv.b : lv.r) : (const Acc*)lv.r32;
  const T* __restrict__ st = static_cast<const T*>(lv.inv);
  int v[3] = {0, 0, 0};
  vertex_of_t<D>(g, p, v);
  const int N = g.N;
  const int64_t N1 = N + 1;
  Acc acc[NROW][NR];
#pragma unroll
  for (int i = 0; i < NROW; ++i)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[i][j] = 0;
  for (int a2 = 0; a2 < (D == 3 ? 3 : 1); ++a2) {
    const int J2 = D == 3 ? v[2] - 1 + a2 : 0;
    const bool ok2 = D == 2 || (J2 >= 1 && J2 <= N - 1);
    for (int a1 = 0; a1 < 3; ++a1) {
      const int J1 = v[1] - 1 + a1;
      const bool ok1 = ok2 && J1 >= 1 && J1 <= N - 1;
#pragma unroll
      for (int a0 = 0; a0 < 3; ++a0) {
        const int n = a0 + 3 * a1 + 9 * a2;
        const int J0 = v[0] - 1 + a0;
        const bool ok = ok1 && J0 >= 1 && J0 <= N - 1;
        const int64_t base = (int64_t)D * (J0 + N1 * (J1 + N1 * J2));
#pragma unroll
        for (int c = 0; c < D; ++c) {
          Acc ra[NR];
          if (ok) {
            load_row<Acc, NR>(r + (base + c) * NR, ra);
          } else {
#pragma unroll
            for (int j = 0; j < NR; ++j) ra[j] = 0;
          }
#pragma unroll
          for (int i = 0; i < NROW; ++i) {
            const Acc q = (Acc)ld_stream(st + ((int64_t)i * NC + n * D + c) * np + p);
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[i][j] += q * ra[j];
          }
        }
      }
    }
  }
  {
    Acc ra[NR];
    load_row<Acc, NR>(r + (g.n_u + p) * NR, ra);
#pragma unroll
    for (int i = 0; i < NROW; ++i) {
      const Acc q = (Acc)ld_stream(st + ((int64_t)i * NC + NC - 1) * np + p);
#pragma unroll
      for (int j = 0; j < NR; ++j) acc[i][j] += q * ra[j];
    }
  }
  const double om = lv.omega[p];
  bool cfree = true;
#pragma unroll
  for (int d = 0; d < D; ++d) cfree &= v[d] >= 1 && v[d] <= N - 1;
  if (cfree) {
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int j = 0; j < NR; ++j) lv.x[((int64_t)D * p + c) * NR + j] += om * (double)acc[c][j];
  }
#pragma unroll
  for (int j = 0; j < NR; ++j) lv.x[(g.n_u + p) * NR + j] += om * (double)acc[D][j];
}

// Q1-Q1 restriction (same order per RHS as k_restrict_q1); zeroes the coarser iterate.
template <int D, int NR>
__global__ void kb_restrict_q1(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne) {
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const Geo &gf = lv.g, &gc = lv.gc;
  const XferTab& T = lv.tab;
  const int t = (int)((blockIdx.x - first[e]) * blockDim.x + threadIdx.x);
  if (t >= (int)gc.n_p) return;
  const int Nf1 = gf.N + 1, Nc1 = gc.N + 1;
  const double* rf = lv.r;
  int K[3] = {0, 0, 0}, id = t;
  bool cbnd = false;
  for (int a = 0; a < D; ++a) {
    K[a] = id % Nc1;
    id /= Nc1;
    cbnd |= (K[a] == 0) | (K[a] == gc.N);
  }
  const int c0 = T.rc1[0][K[0]], c1 = T.rc1[1][K[1]], c2 = D == 3 ? T.rc1[2][K[2]] : 1;
  double acc[D + 1][NR];
#pragma unroll
  for (int c = 0; c <= D; ++c)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[c][j] = 0.0;
  for (int j2 = 0; j2 < c2; ++j2) {
    const int V2 = D == 3 ? T.rk1[2][3 * K[2] + j2] : 0;
    const double w2 = D == 3 ? T.rw1[2][3 * K[2] + j2] : 1.0;
    const bool b2 = D == 3 && (V2 == 0 || V2 == gf.N);
    for (int j1 = 0; j1 < c1; ++j1) {
      const int V1 = T.rk1[1][3 * K[1] + j1];
      const double w12 = D == 3 ? w2 * T.rw1[1][3 * K[1] + j1] : T.rw1[1][3 * K[1] + j1];
      const bool b1 = b2 || V1 == 0 || V1 == gf.N;
#pragma unroll
      for (int j0 = 0; j0 < 3; ++j0)
        if (j0 < c0) {
          const int V0 = T.rk1[0][3 * K[0] + j0];
          const double ww = w12 * T.rw1[0][3 * K[0] + j0];
          const int64_t V = V0 + Nf1 * (V1 + (int64_t)Nf1 * V2);
          if (!(b1 || V0 == 0 || V0 == gf.N)) {
#pragma unroll
            for (int c = 0; c < D; ++c)
#pragma unroll
              for (int j = 0; j < NR; ++j) acc[c][j] += ww * rf[((int64_t)D * V + c) * NR + j];
          }
#pragma unroll
          for (int j = 0; j < NR; ++j) acc[D][j] += ww * rf[(gf.n_u + V) * NR + j];
        }
    }
  }
#pragma unroll
  for (int c = 0; c < D; ++c)
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      const double val = cbnd ? 0.0 : acc[c][j];
      const int64_t o = ((int64_t)D * t + c) * NR + j;
      lv.bc[o] = val;
      if (lv.bc32) lv.bc32[o] = (float)val;
      lv.xc[o] = 0.0;
    }
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    const int64_t o = (gc.n_u + t) * NR + j;
    lv.bc[o] = acc[D][j];
    if (lv.bc32) lv.bc32[o] = (float)acc[D][j];
    lv.xc[o] = 0.0;
  }
}

// Q1-Q1 prolongation x += P xc (same order per RHS as k_prolong_q1).
template <int D, int NR>
__global__ void kb_prolong_q1(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne) {
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const Geo &gf = lv.g, &gc = lv.gc;
  const XferTab& T = lv.tab;
  const int t = (int)((blockIdx.x - first[e]) * blockDim.x + threadIdx.x);
  if (t >= (int)gf.n_p) return;
  const int Nf1 = gf.N + 1, Nc1 = gc.N + 1;
  const double* xc = lv.xc;
  int v[3] = {0, 0, 0}, id = t;
  bool bnd = false;
  for (int a = 0; a < D; ++a) {
    v[a] = id % Nf1;
    id /= Nf1;
    bnd |= (v[a] == 0) | (v[a] == gf.N);
  }
  const int c0 = T.pc1[0][v[0]], c1 = T.pc1[1][v[1]], c2 = D == 3 ? T.pc1[2][v[2]] : 1;
  double acc[D + 1][NR];
#pragma unroll
  for (int c = 0; c <= D; ++c)
#pragma unroll
    for (int j = 0; j < NR; ++j) acc[c][j] = 0.0;
  for (int j2 = 0; j2 < c2; ++j2) {
    const int K2 = D == 3 ? T.pk1[2][2 * v[2] + j2] : 0;
    const double w2 = D == 3 ? T.pw1[2][2 * v[2] + j2] : 1.0;
    for (int j1 = 0; j1 < c1; ++j1) {
      const int K1 = T.pk1[1][2 * v[1] + j1];
      const double w12 = D == 3 ? w2 * T.pw1[1][2 * v[1] + j1] : T.pw1[1][2 * v[1] + j1];
#pragma unroll
      for (int j0 = 0; j0 < 2; ++j0)
        if (j0 < c0) {
          const double ww = w12 * T.pw1[0][2 * v[0] + j0];
          const int K = T.pk1[0][2 * v[0] + j0] + Nc1 * (K1 + Nc1 * K2);
#pragma unroll
          for (int c = 0; c < D; ++c)
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[c][j] += ww * xc[((int64_t)D * K + c) * NR + j];
#pragma unroll
          for (int j = 0; j < NR; ++j) acc[D][j] += ww * xc[(gc.n_u + K) * NR + j];
        }
    }
  }
  if (!bnd) {
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
      for (int j = 0; j < NR; ++j) lv.x[((int64_t)D * t + c) * NR + j] += acc[c][j];
  }
#pragma unroll
  for (int j = 0; j < NR; ++j) lv.x[(gf.n_u + t) * NR + j] += acc[D][j];
}

// Coarse solve on the coarsest level of each entry: r <- b masked to free
// rows, then x = C r (one warp per row, same order per RHS as k_coarse_gemv).
template <int NR>
__global__ void kb_coarse_mask(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne) {
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const int64_t i = (blockIdx.x - first[e]) * (int64_t)blockDim.x + threadIdx.x;
  if (i >= lv.g.n) return;
  const bool d = is_dirichlet(lv.g, i);
#pragma unroll
  for (int j = 0; j < NR; ++j) lv.r[i * NR + j] = d ? 0.0 : lv.b[i * NR + j];
}
template <int NR>
__global__ void kb_coarse_gemv(const BLevel* __restrict__ L, const int64_t* __restrict__ first, int ne) {
  const int e = find_entry(first, ne, blockIdx.x);
  const BLevel& lv = L[e];
  const int64_t n = lv.g.n, m = n + 1;
  const int lane = threadIdx.x & 31;
  const int64_t row = (blockIdx.x - first[e]) * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  double s[NR];
#pragma unroll
  for (int j = 0; j < NR; ++j) s[j] = 0.0;
  for (int64_t c = lane; c < n; c += 32) {
    const double a = lv.cinv[row * m + c];
#pragma unroll
    for (int j = 0; j < NR; ++j) s[j] += a * lv.r[c * NR + j];
  }
#pragma unroll
  for (int j = 0; j < NR; ++j) {
    for (int o = 16; o > 0; o >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
    if (lane == 0) lv.x[row * NR + j] = s[j];
  }
}

}  // namespace rav

using namespace rav;

// One launch: descriptors of the taking-part entries, their block offsets.
struct BPhase {
  BLevel* L = nullptr;      // device
  int64_t* first = nullptr; // device, ne + 1
  int* prob = nullptr;      // device, ne (norm phases)
  int ne = 0, cap = 0;  // entries, allocated descriptor slots
  int64_t blocks = 0;
  int threads = 0;
  std::vector<int> entries;  // host: indices into rav_batch::lv
};

struct rav_batch {
  int nprob = 0, nrhs = 0, dim = 2, prec = RAV_F32, depth = 0;
  int elem = RAV_ELEM_Q2Q1;  // every problem of a batch has the same element
  std::vector<rav_mg*> mgs;
  std::vector<rav_smoother*> sms;
  // host copies of every (problem, level) descriptor, finest level first per problem
  std::vector<BLevel> lv;
  std::vector<int> lv_first;  // start of problem p's levels in lv (finest level of p at lv_first[p])
  std::vector<void*> owned;    // batch-owned vectors
  BLevel* lv_dev = nullptr;    // device mirror of lv
  int tpb_res = 256, tpb_apply = 128;
  // phases per depth d (0 = finest)
  std::vector<BPhase> res_smooth, apply, res_last, restrict_, prolong, coarse_mask, coarse_gemv;
  // shared-inverse tensor-core apply (kb_apply_tc): per depth, the entries
  // whose interior subdomains share their rows; blocks = tiles of 16
  bool use_tc = false;
  // fp32 residuals below the finest depth (batch_set_coarse_residual_f32)
  bool coarse_f32 = false;
  std::vector<void*> c32_bufs;
  // fp32 transfers (batch_set_transfers_f32) and their buffers
  bool xfer_f32 = false;
  std::vector<void*> x32_bufs;
  std::vector<BPhase> tc_apply;
  // tiled apply (kb_apply_tile, 2-D Q2-Q1, fp32 rows, 8 RHS): per depth the
  // rows of vertices per block (2 or 4), 0 where kb_apply runs, and the warps
  // per row of vertices (1 or 2); the set-up tuner's choice is kept in
  // tile_auto / split_auto (batch_set_apply_tile(-1, ...) restores it)
  std::vector<int> tile_ty, tile_auto, tile_split, split_auto;
  std::vector<BPhase> apply_tile;
  std::vector<float*> gtc_bufs;  // per lv entry, null where not shared
  int* tc_err = nullptr;         // set by a tensor-core block whose wait gave up
  BPhase fine_res;  // depth-0 residual with norms
  double* part = nullptr;
  double* norms = nullptr;   // device, nprob * nrhs
  double* norms_h = nullptr; // pinned
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_nu1 = -1, graph_nu2 = -1;
  int64_t graph_launches = 0;
  std::vector<const double*> cur_x, cur_b;
  // timing hook: events around every phase launch while enabled (cycles then
  // run kernel by kernel instead of from the graph)
  bool prof = false;
  struct Ev {
    int depth, kind;
    cudaEvent_t a, b;
  };
  std::vector<Ev> evs;
  size_t ev_used = 0;
  double prof_ms[kMaxLevels][5] = {};
  int64_t prof_cnt[kMaxLevels][5] = {};
};

static int bprof_begin(rav_batch* bt, int depth, int kind, cudaStream_t s) {
  if (!bt->prof) return -1;
  if (bt->ev_used == bt->evs.size()) {
    rav_batch::Ev e{0, 0, nullptr, nullptr};
    if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) return -1;
    bt->evs.push_back(e);
  }
  rav_batch::Ev& e = bt->evs[bt->ev_used];
  e.depth = depth;
  e.kind = kind;
  cudaEventRecord(e.a, s);
  return (int)bt->ev_used++;
}
static void bprof_end(rav_batch* bt, int i, cudaStream_t s) {
  if (i >= 0) cudaEventRecord(bt->evs[i].b, s);
}
static int bprof_collect(rav_batch* bt) {
  for (size_t i = 0; i < bt->ev_used; ++i) {
    rav_batch::Ev& e = bt->evs[i];
    float ms = 0.0f;
    RAV_CUDA(cudaEventSynchronize(e.b));
    RAV_CUDA(cudaEventElapsedTime(&ms, e.a, e.b));
    bt->prof_ms[e.depth][e.kind] += ms;
    bt->prof_cnt[e.depth][e.kind] += 1;
  }
  bt->ev_used = 0;
  return RAV_OK;
}

static int level_count(const rav_batch* bt, int p) {
  return bt->mgs[p]->nlev;
}

// Builds the descriptor of problem p at depth d (level nlev-1-d).
static BLevel make_level(rav_batch* bt, int p, int d) {
  rav_mg* mg = bt->mgs[p];
  rav_smoother* sm = bt->sms[p];
  const int l = mg->nlev - 1 - d;
  const Level& L = mg->lev[l];
  BLevel b{};
  b.g = L.g;
  if (l > 0) b.gc = mg->lev[l - 1].g;
  b.nslice = L.nslice;
  b.sperm = L.sperm;
  b.sptr = L.sptr;
  b.slen = L.slen;
  b.scol = L.scol;
  b.sval = L.sval;
  if (l > 0) {
    b.inv = sm->lev[l].inv;
    b.omega = sm->lev[l].omega;
    b.units = sm->lev[l].units;
    b.tab = L.tab();
  }
  b.cinv = l == 0 ? mg->cinv : nullptr;
  b.problem = p;
  return b;
}

static int upload_phase(rav_batch* bt, BPhase& ph, const std::vector<int>& entries, int threads,
                        int64_t (*blocks_of)(const BLevel&, int)) {
  ph.entries = entries;
  ph.ne = (int)entries.size();
  ph.threads = threads;
  if (ph.ne == 0) return RAV_OK;
  std::vector<BLevel> h(ph.ne);
  std::vector<int64_t> first(ph.ne + 1, 0);
  std::vector<int> prob(ph.ne);
  for (int i = 0; i < ph.ne; ++i) {
    h[i] = bt->lv[entries[i]];
    prob[i] = h[i].problem;
    first[i + 1] = first[i] + blocks_of(h[i], threads);
  }
  ph.blocks = first[ph.ne];
  if (ph.ne > ph.cap) {
    cudaFree(ph.L);
    cudaFree(ph.first);
    cudaFree(ph.prob);
    ph.L = nullptr;
    ph.first = nullptr;
    ph.prob = nullptr;
    RAV_CUDA(cudaMalloc(&ph.L, sizeof(BLevel) * ph.ne));
    RAV_CUDA(cudaMalloc(&ph.first, sizeof(int64_t) * (ph.ne + 1)));
    RAV_CUDA(cudaMalloc(&ph.prob, sizeof(int) * ph.ne));
    ph.cap = ph.ne;
  }
  RAV_CUDA(cudaMemcpy(ph.L, h.data(), sizeof(BLevel) * ph.ne, cudaMemcpyHostToDevice));
  RAV_CUDA(cudaMemcpy(ph.first, first.data(), sizeof(int64_t) * (ph.ne + 1), cudaMemcpyHostToDevice));
  RAV_CUDA(cudaMemcpy(ph.prob, prob.data(), sizeof(int) * ph.ne, cudaMemcpyHostToDevice));
  return RAV_OK;
}

static int64_t blk_res(const BLevel& b, int t) { return (b.nslice * 32 + t - 1) / t; }
static int64_t blk_apply(const BLevel& b, int t) { return (b.units + t - 1) / t; }
static int64_t blk_restrict(const BLevel& b, int t) {
  if (b.g.q == 1) return (b.gc.n_p + t - 1) / t;
  return ((b.gc.nnode + b.gc.n_p) * restrict_split(b.gc) + t - 1) / t;
}
static int64_t blk_prolong(const BLevel& b, int t) {
  return ((b.g.q == 1 ? 0 : b.g.nnode) + b.g.n_p + t - 1) / t;
}
static int64_t blk_mask(const BLevel& b, int t) { return (b.g.n + t - 1) / t; }
static int64_t blk_tc(const BLevel& b, int) {
  const int64_t ni = b.g.N - 3;
  return (ni * ni + kTcP - 1) / kTcP;
}
static int64_t blk_gemv(const BLevel& b, int t) { return (b.g.n + t / 32 - 1) / (t / 32); }
template <int SPLIT>  // threads t = 32 x TY x SPLIT
static int64_t blk_tile(const BLevel& b, int t) {
  const int64_t v = b.g.N + 1, ty = t / (kTileX * SPLIT);
  return (v + kTileX - 1) / kTileX * ((v + ty - 1) / ty);
}
static bool tile_ok(const rav_batch* bt) {
  return bt->dim == 2 && bt->nrhs == 8 && bt->prec == RAV_F32 && bt->elem == RAV_ELEM_Q2Q1;
}

// ---- launches --------------------------------------------------------------
template <int NR>
static void launch_res(const BPhase& ph, double* part, cudaStream_t s, bool f32 = false) {
  if (!ph.ne) return;
  if (f32) {  // no norm partials on these depths
    kb_x_to_f32<NR><<<(unsigned)ph.blocks, ph.threads, 0, s>>>(ph.L, ph.first, ph.ne);
    kb_residual_f32<NR><<<(unsigned)ph.blocks, ph.threads, 0, s>>>(ph.L, ph.first, ph.ne);
  } else {
    kb_residual<NR><<<(unsigned)ph.blocks, ph.threads, 0, s>>>(ph.L, ph.first, ph.ne, part);
  }
}
template <int D, int NR>
static void launch_apply(const rav_batch* bt, const BPhase& ph, int use_b, cudaStream_t s) {
  if (!ph.ne) return;
  if (bt->elem == RAV_ELEM_Q1Q1) {
    if (bt->prec == RAV_F32)
      kb_apply_q1<D, float, NR><<<(unsigned)ph.blocks, ph.threads, 0, s>>>(ph.L, ph.first, ph.ne, use_b);
    else
      kb_apply_q1<D, double, NR><<<(unsigned)ph.blocks, ph.threads, 0, s>>>(ph.L, ph.first, ph.ne, use_b);
  } else if (bt->prec == RAV_F32) {
    kb_apply<D, float, NR><<<(unsigned)ph.blocks, ph.threads, 0, s>>>(ph.L, ph.first, ph.ne, use_b);
  } else {
    kb_apply<D, double, NR><<<(unsigned)ph.blocks, ph.threads, 0, s>>>(ph.L, ph.first, ph.ne, use_b);
  }
}

static void launch_tile(const BPhase& ph, int ty, int split, cudaStream_t s) {
  if (!ph.ne) return;
  const unsigned nb = (unsigned)ph.blocks;
  if (ty == 2 && split == 1) kb_apply_tile<2, 1><<<nb, ph.threads, 0, s>>>(ph.L, ph.first, ph.ne);
  else if (ty == 4 && split == 1) kb_apply_tile<4, 1><<<nb, ph.threads, 0, s>>>(ph.L, ph.first, ph.ne);
  else if (ty == 2) kb_apply_tile<2, 2><<<nb, ph.threads, 0, s>>>(ph.L, ph.first, ph.ne);
  else kb_apply_tile<4, 2><<<nb, ph.threads, 0, s>>>(ph.L, ph.first, ph.ne);
}

template <int D, int NR>
static int batch_cycle(rav_batch* bt, int nu1, int nu2, cudaStream_t s) {
  const int Dm = bt->depth;
  int ev;
  auto res = [&](int d) {
    ev = bprof_begin(bt, d, PROF_RESIDUAL, s);
    launch_res<NR>(bt->res_smooth[d], nullptr, s, bt->coarse_f32 && d > 0);
    bprof_end(bt, ev, s);
  };
  auto apply = [&](int d, int use_b) {
    ev = bprof_begin(bt, d, PROF_APPLY, s);
    if (d < (int)bt->tile_ty.size() && bt->tile_ty[d])  // fp32 rows: reads r32 either way
      launch_tile(bt->apply_tile[d], bt->tile_ty[d], bt->tile_split[d], s);
    else
      launch_apply<D, NR>(bt, bt->apply[d], use_b, s);
    if (bt->use_tc && d < (int)bt->tc_apply.size() && bt->tc_apply[d].ne) {
      const BPhase& tp = bt->tc_apply[d];
      const unsigned grid = (unsigned)std::min<int64_t>(tp.blocks, 152 * 2);
      kb_apply_tc<<<grid, 256, kTcSmem, s>>>(tp.L, tp.first, tp.ne, bt->tc_err);
    }
    bprof_end(bt, ev, s);
  };
  // down
  for (int d = 0; d < Dm; ++d) {
    for (int it = 0; it < nu1; ++it) {
      if (it == 0 && d > 0) {
        apply(d, 1);
      } else {
        res(d);
        apply(d, 0);
      }
    }
    res(d);
    const BPhase& rp = bt->restrict_[d];
    ev = bprof_begin(bt, d, PROF_RESTRICT, s);
    if (rp.ne && bt->elem == RAV_ELEM_Q1Q1)
      kb_restrict_q1<D, NR><<<(unsigned)rp.blocks, rp.threads, 0, s>>>(rp.L, rp.first, rp.ne);
    else if (rp.ne && bt->xfer_f32)
      kb_restrict<D, NR, float><<<(unsigned)rp.blocks, rp.threads, 0, s>>>(rp.L, rp.first, rp.ne);
    else if (rp.ne)
      kb_restrict<D, NR, double><<<(unsigned)rp.blocks, rp.threads, 0, s>>>(rp.L, rp.first, rp.ne);
    bprof_end(bt, ev, s);
    const BPhase& cm = bt->coarse_mask[d + 1];
    if (cm.ne) {
      ev = bprof_begin(bt, d + 1, PROF_COARSE, s);
      kb_coarse_mask<NR><<<(unsigned)cm.blocks, cm.threads, 0, s>>>(cm.L, cm.first, cm.ne);
      const BPhase& cg = bt->coarse_gemv[d + 1];
      kb_coarse_gemv<NR><<<(unsigned)cg.blocks, cg.threads, 0, s>>>(cg.L, cg.first, cg.ne);
      bprof_end(bt, ev, s);
    }
  }
  // up
  for (int d = Dm - 1; d >= 0; --d) {
    const BPhase& pp = bt->prolong[d];
    ev = bprof_begin(bt, d, PROF_PROLONG, s);
    if (pp.ne && bt->elem == RAV_ELEM_Q1Q1) {
      kb_prolong_q1<D, NR><<<(unsigned)pp.blocks, pp.threads, 0, s>>>(pp.L, pp.first, pp.ne);
    } else if (pp.ne && bt->xfer_f32) {
      kb_xc_to_f32<NR><<<(unsigned)pp.blocks, pp.threads, 0, s>>>(pp.L, pp.first, pp.ne);
      kb_prolong<D, NR, float><<<(unsigned)pp.blocks, pp.threads, 0, s>>>(pp.L, pp.first, pp.ne);
    } else if (pp.ne) {
      kb_prolong<D, NR, double><<<(unsigned)pp.blocks, pp.threads, 0, s>>>(pp.L, pp.first, pp.ne);
    }
    bprof_end(bt, ev, s);
    for (int it = 0; it < nu2; ++it) {
      res(d);
      apply(d, 0);
    }
  }
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

static int batch_cycle_any(rav_batch* bt, int nu1, int nu2, cudaStream_t s) {
  const int D = bt->dim, NR = bt->nrhs;
#define RAV_BC(DD, RR) \
  if (D == DD && NR == RR) return batch_cycle<DD, RR>(bt, nu1, nu2, s);
  RAV_BC(2, 1) RAV_BC(2, 2) RAV_BC(2, 4) RAV_BC(2, 8) RAV_BC(3, 1) RAV_BC(3, 2) RAV_BC(3, 4) RAV_BC(3, 8)
#undef RAV_BC
  return RAV_ERR_ARG;
}

static int fine_norms(rav_batch* bt, cudaStream_t s) {
  const BPhase& ph = bt->fine_res;
  switch (bt->nrhs) {
    case 1: launch_res<1>(ph, bt->part, s); kb_norm_final<1><<<(ph.ne + 127) / 128, 128, 0, s>>>(ph.first, ph.prob, ph.ne, bt->part, bt->norms); break;
    case 2: launch_res<2>(ph, bt->part, s); kb_norm_final<2><<<(ph.ne * 2 + 127) / 128, 128, 0, s>>>(ph.first, ph.prob, ph.ne, bt->part, bt->norms); break;
    case 4: launch_res<4>(ph, bt->part, s); kb_norm_final<4><<<(ph.ne * 4 + 127) / 128, 128, 0, s>>>(ph.first, ph.prob, ph.ne, bt->part, bt->norms); break;
    default: launch_res<8>(ph, bt->part, s); kb_norm_final<8><<<(ph.ne * 8 + 127) / 128, 128, 0, s>>>(ph.first, ph.prob, ph.ne, bt->part, bt->norms); break;
  }
  note_launch(2);
  RAV_CUDA(cudaGetLastError());
  RAV_CUDA(cudaMemcpyAsync(bt->norms_h, bt->norms, sizeof(double) * bt->nprob * bt->nrhs, cudaMemcpyDeviceToHost, s));
  if (bt->use_tc)  // the tensor-core apply's bounded waits report here
    RAV_CUDA(cudaMemcpyAsync(bt->norms_h + bt->nprob * bt->nrhs, bt->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  RAV_CUDA(cudaStreamSynchronize(s));
  if (bt->use_tc && *reinterpret_cast<const int*>(bt->norms_h + bt->nprob * bt->nrhs)) return RAV_ERR_TIMEOUT;
  return RAV_OK;
}

// Builds every phase for the current threads-per-block choices.
static int build_phases(rav_batch* bt) {
  const int Dm = bt->depth;
  bt->res_smooth.resize(Dm);
  bt->apply.resize(Dm);
  bt->restrict_.resize(Dm);
  bt->prolong.resize(Dm);
  bt->coarse_mask.resize(Dm + 1);
  bt->coarse_gemv.resize(Dm + 1);
  for (int d = 0; d <= Dm; ++d) {
    std::vector<int> smooth, coarse;
    for (int p = 0; p < bt->nprob; ++p) {
      const int Lp = level_count(bt, p);
      if (d <= Lp - 2) smooth.push_back(bt->lv_first[p] + d);
      if (d == Lp - 1) coarse.push_back(bt->lv_first[p] + d);
    }
    if (d < Dm) {
      RAV_TRY(upload_phase(bt, bt->res_smooth[d], smooth, bt->tpb_res, blk_res));
      RAV_TRY(upload_phase(bt, bt->apply[d], smooth, bt->tpb_apply, blk_apply));
      RAV_TRY(upload_phase(bt, bt->restrict_[d], smooth, 128, blk_restrict));
      RAV_TRY(upload_phase(bt, bt->prolong[d], smooth, 128, blk_prolong));
    }
    RAV_TRY(upload_phase(bt, bt->coarse_mask[d], coarse, 256, blk_mask));
    RAV_TRY(upload_phase(bt, bt->coarse_gemv[d], coarse, 256, blk_gemv));
  }
  bt->apply_tile.resize(Dm);
  for (int d = 0; d < Dm; ++d) {
    const int ty = d < (int)bt->tile_ty.size() ? bt->tile_ty[d] : 0;
    const int sp = ty ? bt->tile_split[d] : 1;
    RAV_TRY(upload_phase(bt, bt->apply_tile[d], ty ? bt->apply[d].entries : std::vector<int>{},
                         kTileX * (ty ? ty : 2) * sp, sp == 2 ? blk_tile<2> : blk_tile<1>));
  }
  bt->tc_apply.resize(Dm);
  for (int d = 0; d < Dm; ++d) {
    std::vector<int> shared;
    for (int p = 0; p < bt->nprob; ++p)
      if (d <= level_count(bt, p) - 2 && bt->lv[bt->lv_first[p] + d].gtc) shared.push_back(bt->lv_first[p] + d);
    RAV_TRY(upload_phase(bt, bt->tc_apply[d], shared, 256, blk_tc));
  }
  std::vector<int> fine;
  for (int p = 0; p < bt->nprob; ++p) fine.push_back(bt->lv_first[p]);
  RAV_TRY(upload_phase(bt, bt->fine_res, fine, 256, blk_res));
  if (bt->part) cudaFree(bt->part);
  RAV_CUDA(cudaMalloc(&bt->part, sizeof(double) * (bt->fine_res.blocks + 1) * bt->nrhs));
  return RAV_OK;
}

// Points the finest-level descriptors at the caller's vectors.
static int bind_vectors(rav_batch* bt, double* const* x, const double* const* b) {
  bool same = (int)bt->cur_x.size() == bt->nprob;
  for (int p = 0; same && p < bt->nprob; ++p) same = bt->cur_x[p] == x[p] && bt->cur_b[p] == b[p];
  if (same) return RAV_OK;
  bt->cur_x.assign(x, x + bt->nprob);
  bt->cur_b.assign(b, b + bt->nprob);
  for (int p = 0; p < bt->nprob; ++p) {
    BLevel& f = bt->lv[bt->lv_first[p]];
    f.x = x[p];
    f.b = const_cast<double*>(b[p]);
  }
  // re-upload the descriptors of every phase (they hold copies)
  std::vector<BPhase*> all;
  for (auto* v : {&bt->res_smooth, &bt->apply, &bt->restrict_, &bt->prolong, &bt->coarse_mask, &bt->coarse_gemv,
                  &bt->tc_apply, &bt->apply_tile})
    for (auto& ph : *v) all.push_back(&ph);
  all.push_back(&bt->fine_res);
  for (BPhase* ph : all) {
    if (!ph->ne) continue;
    std::vector<BLevel> h(ph->ne);
    for (int i = 0; i < ph->ne; ++i) h[i] = bt->lv[ph->entries[i]];
    RAV_CUDA(cudaMemcpy(ph->L, h.data(), sizeof(BLevel) * ph->ne, cudaMemcpyHostToDevice));
  }
  return RAV_OK;
}

// Autotuner: times the finest-depth residual and apply phases for each
// candidate block size on the batch's own data and keeps the fastest.
static int autotune(rav_batch* bt, cudaStream_t s) {
  cudaEvent_t e0, e1;
  RAV_CUDA(cudaEventCreate(&e0));
  RAV_CUDA(cudaEventCreate(&e1));
  auto time_it = [&](auto&& fn) -> float {
    fn();
    cudaEventRecord(e0, s);
    for (int i = 0; i < 3; ++i) fn();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  const int cand_res[3] = {128, 256, 512}, cand_apply[3] = {64, 128, 256};
  float best = 1e30f;
  int bres = 256, bapp = 128;
  for (int c : cand_res) {
    bt->tpb_res = c;
    RAV_TRY(build_phases(bt));
    const float ms = time_it([&] {
      switch (bt->nrhs) {
        case 1: launch_res<1>(bt->res_smooth[0], nullptr, s); break;
        case 2: launch_res<2>(bt->res_smooth[0], nullptr, s); break;
        case 4: launch_res<4>(bt->res_smooth[0], nullptr, s); break;
        default: launch_res<8>(bt->res_smooth[0], nullptr, s); break;
      }
    });
    if (ms < best) { best = ms; bres = c; }
  }
  bt->tpb_res = bres;
  best = 1e30f;
  std::vector<double> xsave;
  for (int c : cand_apply) {
    bt->tpb_apply = c;
    RAV_TRY(build_phases(bt));
    // the apply updates x; time on the batch's own level-1 work vectors when
    // they exist, else on the caller-free finest data with x restored below
    const float ms = time_it([&] {
      if (bt->dim == 2) {
        switch (bt->nrhs) {
          case 1: launch_apply<2, 1>(bt, bt->apply[0], 0, s); break;
          case 2: launch_apply<2, 2>(bt, bt->apply[0], 0, s); break;
          case 4: launch_apply<2, 4>(bt, bt->apply[0], 0, s); break;
          default: launch_apply<2, 8>(bt, bt->apply[0], 0, s); break;
        }
      } else {
        switch (bt->nrhs) {
          case 1: launch_apply<3, 1>(bt, bt->apply[0], 0, s); break;
          case 2: launch_apply<3, 2>(bt, bt->apply[0], 0, s); break;
          case 4: launch_apply<3, 4>(bt, bt->apply[0], 0, s); break;
          default: launch_apply<3, 8>(bt, bt->apply[0], 0, s); break;
        }
      }
    });
    if (ms < best) { best = ms; bapp = c; }
  }
  bt->tpb_apply = bapp;
  // per depth: kb_apply or the tiled apply with 2 or 4 rows of vertices per
  // block (one warp per row wastes lanes where a level has few vertices)
  bt->tile_ty.assign(bt->depth, 0);
  bt->tile_split.assign(bt->depth, 1);
  if (tile_ok(bt)) {
    RAV_TRY(build_phases(bt));
    for (int d = 0; d < bt->depth; ++d) {
      if (!bt->apply[d].ne) continue;
      float bd = time_it([&] { launch_apply<2, 8>(bt, bt->apply[d], 0, s); });
      for (int sp : {1, 2})
        for (int ty : {2, 4}) {
          BPhase tmp;
          int rc = upload_phase(bt, tmp, bt->apply[d].entries, kTileX * ty * sp, sp == 2 ? blk_tile<2> : blk_tile<1>);
          const float ms = rc == RAV_OK ? time_it([&] { launch_tile(tmp, ty, sp, s); }) : 1e30f;
          cudaFree(tmp.L);
          cudaFree(tmp.first);
          cudaFree(tmp.prob);
          RAV_TRY(rc);
          if (ms < bd) {
            bd = ms;
            bt->tile_ty[d] = ty;
            bt->tile_split[d] = sp;
          }
        }
    }
  }
  bt->tile_auto = bt->tile_ty;
  bt->split_auto = bt->tile_split;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  RAV_TRY(build_phases(bt));
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

extern "C" int batch_setup(rav_mg* const* mgs, rav_smoother* const* sms, int nprob, int nrhs, rav_stream stream,
                           rav_batch** out) {
  if (!mgs || !sms || !out || nprob < 1 || !(nrhs == 1 || nrhs == 2 || nrhs == 4 || nrhs == 8)) return RAV_ERR_ARG;
  *out = nullptr;
  const int dim = mgs[0] ? mgs[0]->dim : 0;
  const int prec = sms[0] ? sms[0]->prec : -1;
  for (int p = 0; p < nprob; ++p) {
    if (!mgs[p] || !sms[p] || sms[p]->mg != mgs[p] || mgs[p]->dim != dim || mgs[p]->nlev < 2) return RAV_ERR_ARG;
    if (sms[p]->kind != RAV_RAV || sms[p]->prec != prec) return RAV_ERR_ARG;
    if (mgs[p]->elem != mgs[0]->elem) return RAV_ERR_ARG;  // one element per batch
  }
  if (prec != RAV_F32 && prec != RAV_F64_ROWS) return RAV_ERR_ARG;
  cudaStream_t s = S(stream);
  rav_batch* bt = new rav_batch();
  bt->nprob = nprob;
  bt->nrhs = nrhs;
  bt->dim = dim;
  bt->prec = prec;
  bt->elem = mgs[0]->elem;
  bt->mgs.assign(mgs, mgs + nprob);
  bt->sms.assign(sms, sms + nprob);
  auto fail = [&](int rc) {
    batch_destroy(bt);
    return rc;
  };
  // descriptors and batch-owned vectors (every level of every problem, finest first)
  for (int p = 0; p < nprob; ++p) {
    bt->lv_first.push_back((int)bt->lv.size());
    const int Lp = mgs[p]->nlev;
    bt->depth = std::max(bt->depth, Lp - 1);
    for (int d = 0; d < Lp; ++d) bt->lv.push_back(make_level(bt, p, d));
    for (int d = 0; d < Lp; ++d) {
      BLevel& b = bt->lv[bt->lv_first[p] + d];
      const int64_t n = b.g.n * nrhs;
      double* v[3] = {nullptr, nullptr, nullptr};
      for (int k = (d == 0 ? 2 : 0); k < 3; ++k) {
        if (cudaMalloc(&v[k], sizeof(double) * n) != cudaSuccess) return fail(RAV_ERR_CUDA);
        cudaMemset(v[k], 0, sizeof(double) * n);
        bt->owned.push_back(v[k]);
      }
      if (d > 0) { b.x = v[0]; b.b = v[1]; }
      b.r = v[2];
      b.r32 = nullptr;
      if (prec == RAV_F32 && d + 1 < Lp) {  // the coarsest level is solved directly
        float* f = nullptr;
        if (cudaMalloc(&f, sizeof(float) * n) != cudaSuccess) return fail(RAV_ERR_CUDA);
        cudaMemset(f, 0, sizeof(float) * n);
        bt->owned.push_back(f);
        b.r32 = f;
      }
    }
    for (int d = 0; d < Lp; ++d) {
      BLevel& b = bt->lv[bt->lv_first[p] + d];
      b.xc = d + 1 < Lp ? bt->lv[bt->lv_first[p] + d + 1].x : nullptr;
      b.bc = d + 1 < Lp ? bt->lv[bt->lv_first[p] + d + 1].b : nullptr;
      b.bc32 = d + 1 < Lp ? bt->lv[bt->lv_first[p] + d + 1].r32 : nullptr;
    }
  }
  // the finest x, b are bound per call; give them scratch for the autotuner
  for (int p = 0; p < nprob; ++p) {
    BLevel& f = bt->lv[bt->lv_first[p]];
    const int64_t n = f.g.n * nrhs;
    double *x = nullptr, *b = nullptr;
    if (cudaMalloc(&x, sizeof(double) * n) != cudaSuccess) return fail(RAV_ERR_CUDA);
    if (cudaMalloc(&b, sizeof(double) * n) != cudaSuccess) return fail(RAV_ERR_CUDA);
    cudaMemset(x, 0, sizeof(double) * n);
    cudaMemset(b, 0, sizeof(double) * n);
    bt->owned.push_back(x);
    bt->owned.push_back(b);
    f.x = x;
    f.b = b;
  }
  if (cudaMalloc(&bt->norms, sizeof(double) * nprob * nrhs) != cudaSuccess) return fail(RAV_ERR_CUDA);
  // one spare slot: the tensor-core apply's error flag is read back beside the norms
  if (cudaMallocHost(&bt->norms_h, sizeof(double) * (nprob * nrhs + 1)) != cudaSuccess) return fail(RAV_ERR_CUDA);
  int rc = autotune(bt, s);
  if (rc != RAV_OK) return fail(rc);
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(RAV_ERR_CUDA);
  *out = bt;
  return RAV_OK;
}

extern "C" void batch_destroy(rav_batch* bt) {
  if (!bt) return;
  cudaDeviceSynchronize();
  if (bt->graph) cudaGraphExecDestroy(bt->graph);
  if (bt->cap) cudaStreamDestroy(bt->cap);
  for (void* q : bt->c32_bufs) cudaFree(q);
  for (void* q : bt->x32_bufs) cudaFree(q);
  for (auto& e : bt->evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto* v : {&bt->res_smooth, &bt->apply, &bt->restrict_, &bt->prolong, &bt->coarse_mask, &bt->coarse_gemv,
                  &bt->tc_apply, &bt->apply_tile})
    for (auto& ph : *v) {
      cudaFree(ph.L);
      cudaFree(ph.first);
      cudaFree(ph.prob);
    }
  for (float* g : bt->gtc_bufs) cudaFree(g);
  cudaFree(bt->tc_err);
  cudaFree(bt->fine_res.L);
  cudaFree(bt->fine_res.first);
  cudaFree(bt->fine_res.prob);
  for (void* p : bt->owned) cudaFree(p);
  cudaFree(bt->part);
  cudaFree(bt->norms);
  if (bt->norms_h) cudaFreeHost(bt->norms_h);
  delete bt;
}

extern "C" int batch_set_apply_tile(rav_batch* bt, int ty, int split, rav_stream stream) {
  if (!bt || !(ty == -1 || ty == 0 || ty == 2 || ty == 4) || !(split == 1 || split == 2)) return RAV_ERR_ARG;
  if (ty > 0 && !tile_ok(bt)) return RAV_ERR_ARG;
  cudaStream_t s = S(stream);
  RAV_CUDA(cudaStreamSynchronize(s));
  if (ty < 0) {
    bt->tile_ty = bt->tile_auto;
    bt->tile_split = bt->split_auto;
  } else {
    bt->tile_ty.assign(bt->depth, ty);
    bt->tile_split.assign(bt->depth, split);
  }
  if (bt->graph) {  // the captured cycle holds the previous apply kernels
    cudaGraphExecDestroy(bt->graph);
    bt->graph = nullptr;
  }
  bt->cur_x.clear();  // descriptors are re-uploaded at the next bind
  RAV_TRY(build_phases(bt));
  RAV_CUDA(cudaStreamSynchronize(s));
  return RAV_OK;
}

extern "C" int batch_get_apply_tile(const rav_batch* bt, int depth, int out[2]) {
  if (!bt || !out || depth < 0 || depth >= bt->depth) return RAV_ERR_ARG;
  const bool t = depth < (int)bt->tile_ty.size() && bt->tile_ty[depth];
  out[0] = t ? bt->tile_ty[depth] : 0;
  out[1] = t ? bt->tile_split[depth] : 1;
  return RAV_OK;
}

extern "C" int batch_get_tuning(const rav_batch* bt, int out[2]) {
  if (!bt || !out) return RAV_ERR_ARG;
  out[0] = bt->tpb_res;
  out[1] = bt->tpb_apply;
  return RAV_OK;
}

// One batched V-cycle, captured into a graph on first use and replayed.
static int batch_vcycle_impl(rav_batch* bt, int nu1, int nu2, cudaStream_t s) {
  if (bt->prof) {  // kernel by kernel, events around each phase
    const int64_t l0 = rav_kernel_launches();
    RAV_TRY(batch_cycle_any(bt, nu1, nu2, s));
    (void)l0;
    return RAV_OK;
  }
  if (!bt->graph || bt->graph_nu1 != nu1 || bt->graph_nu2 != nu2) {
    if (bt->graph) {
      cudaGraphExecDestroy(bt->graph);
      bt->graph = nullptr;
    }
    if (!bt->cap) RAV_CUDA(cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking));
    const int64_t l0 = rav_kernel_launches();
    RAV_CUDA(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
    const int rc = batch_cycle_any(bt, nu1, nu2, bt->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(bt->cap, &g);
    if (rc != RAV_OK || ec != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return rc != RAV_OK ? rc : RAV_ERR_CUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&bt->graph, g, 0);
    size_t nnodes = 0;
    cudaGraphGetNodes(g, nullptr, &nnodes);
    cudaGraphDestroy(g);
    RAV_CUDA(ei);
    bt->graph_nu1 = nu1;
    bt->graph_nu2 = nu2;
    bt->graph_launches = (int64_t)nnodes;
    (void)l0;
  }
  RAV_CUDA(cudaGraphLaunch(bt->graph, s));
  note_launch((int)bt->graph_launches);
  return RAV_OK;
}

extern "C" int batch_profile_enable(rav_batch* bt, int on) {
  if (!bt) return RAV_ERR_ARG;
  RAV_CUDA(cudaDeviceSynchronize());
  bt->prof = on != 0;
  bt->ev_used = 0;
  for (int d = 0; d < kMaxLevels; ++d)
    for (int k = 0; k < 5; ++k) {
      bt->prof_ms[d][k] = 0.0;
      bt->prof_cnt[d][k] = 0;
    }
  return RAV_OK;
}

extern "C" int batch_profile_read(rav_batch* bt, int depth, int kind, int64_t* launches, double* total_ms) {
  if (!bt || depth < 0 || depth >= kMaxLevels || kind < 0 || kind > 4 || !launches || !total_ms)
    return RAV_ERR_ARG;
  RAV_TRY(bprof_collect(bt));
  *launches = bt->prof_cnt[depth][kind];
  *total_ms = bt->prof_ms[depth][kind];
  return RAV_OK;
}

// The kernels read a row's nrhs values of x and b two doubles at a time when
// nrhs >= 2, so those vectors must start on a 16-byte boundary.
static bool bvec_ok(const rav_batch* bt, const void* v) {
  return v && (bt->nrhs == 1 || (reinterpret_cast<uintptr_t>(v) & 15) == 0);
}

extern "C" int batch_vcycle(rav_batch* bt, double* const* x, const double* const* b, int nu1, int nu2,
                            rav_stream stream) {
  if (!bt || !x || !b || nu1 < 0 || nu2 < 0) return RAV_ERR_ARG;
  for (int p = 0; p < bt->nprob; ++p)
    if (!bvec_ok(bt, x[p]) || !bvec_ok(bt, b[p])) return RAV_ERR_ARG;
  cudaStream_t s = S(stream);
  RAV_CUDA(cudaStreamSynchronize(s));  // descriptors are rewritten below
  RAV_TRY(bind_vectors(bt, x, b));
  return batch_vcycle_impl(bt, nu1, nu2, s);
}

extern "C" int solve_batched(rav_batch* bt, double* const* x, const double* const* b, const rav_solve_opts* o,
                             int* iters, double* ratios, rav_stream stream) {
  if (!bt || !x || !b || !o || o->maxit < 0 || !(o->tol > 0) || o->outer != 0) return RAV_ERR_ARG;
  for (int p = 0; p < bt->nprob; ++p)
    if (!bvec_ok(bt, x[p]) || !bvec_ok(bt, b[p])) return RAV_ERR_ARG;
  cudaStream_t s = S(stream);
  RAV_CUDA(cudaStreamSynchronize(s));
  RAV_TRY(bind_vectors(bt, x, b));
  const int nk = bt->nprob * bt->nrhs;
  std::vector<double> r0(nk);
  std::vector<int> it(nk, -1);
  RAV_TRY(fine_norms(bt, s));
  for (int i = 0; i < nk; ++i) {
    r0[i] = bt->norms_h[i];
    if (r0[i] == 0.0) it[i] = 0;
  }
  std::vector<double> ratio(nk, 1.0);
  int rc = RAV_OK;
  for (int k = 1; k <= o->maxit; ++k) {
    bool all = true;
    for (int i = 0; i < nk; ++i) all &= it[i] >= 0;
    if (all) break;
    RAV_TRY(batch_vcycle_impl(bt, o->nu_pre, o->nu_post, s));
    RAV_TRY(fine_norms(bt, s));
    for (int i = 0; i < nk; ++i) {
      if (it[i] >= 0 || r0[i] == 0.0) continue;
      ratio[i] = bt->norms_h[i] / r0[i];
      if (!std::isfinite(ratio[i])) rc = RAV_ERR_NAN;
      else if (ratio[i] <= o->tol) it[i] = k;
    }
    if (rc != RAV_OK) break;
  }
  bool all = true;
  for (int i = 0; i < nk; ++i) all &= it[i] >= 0;
  if (rc == RAV_OK && !all) rc = RAV_ERR_NOT_CONVERGED;
  for (int i = 0; i < nk; ++i) {
    if (iters) iters[i] = it[i];
    if (ratios) ratios[i] = ratio[i];
  }
  return rc;
}

extern "C" int batch_set_tensor_apply(rav_batch* bt, int enable, rav_stream stream) {
  if (!bt) return RAV_ERR_ARG;
  if (!enable) {
    if (!bt->use_tc) return RAV_OK;
    RAV_CUDA(cudaDeviceSynchronize());
    bt->use_tc = false;
    for (BLevel& b : bt->lv) b.gtc = nullptr;
  } else {
    if (bt->dim != 2 || bt->elem != RAV_ELEM_Q2Q1 || bt->prec != RAV_F32 || bt->nrhs != 8) return RAV_ERR_ARG;
    if (bt->use_tc) return RAV_OK;
    cudaStream_t s = S(stream);
    RAV_CUDA(cudaStreamSynchronize(s));
    if (!bt->tc_err) RAV_CUDA(cudaMalloc(&bt->tc_err, sizeof(int)));
    RAV_CUDA(cudaMemset(bt->tc_err, 0, sizeof(int)));
    RAV_CUDA(cudaFuncSetAttribute(kb_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
    bt->gtc_bufs.resize(bt->lv.size(), nullptr);
    int* bad = nullptr;
    RAV_CUDA(cudaMalloc(&bad, sizeof(int)));
    std::vector<float> h(2048);
    for (size_t i = 0; i < bt->lv.size(); ++i) {
      BLevel& b = bt->lv[i];
      b.gtc = nullptr;
      if (!b.inv || b.g.N < 4) continue;  // coarsest levels, grids without an interior subdomain
      float*& buf = bt->gtc_bufs[i];
      if (!buf && cudaMalloc(&buf, sizeof(float) * 2048) != cudaSuccess) {
        cudaFree(bad);
        return RAV_ERR_CUDA;
      }
      kb_shared_build<<<8, 128, 0, s>>>(b.g, (const float*)b.inv, buf);
      if (cudaMemcpyAsync(h.data(), buf, sizeof(float) * 2048, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(bad);
        return RAV_ERR_CUDA;
      }
      float amax = 0.f;
      for (int k = 0; k < 1024; ++k) amax = std::max(amax, std::fabs(h[k] + h[1024 + k]));
      // stored fp32 rows equal to within two units in the last place of the largest
      const float tol = std::ldexp(amax, -22);
      const int64_t ni = b.g.N - 3, tot = ni * ni * 9 * 51;
      cudaMemsetAsync(bad, 0, sizeof(int), s);
      kb_shared_check<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(b.g, (const float*)b.inv, tol, bad);
      int hb = 1;
      if (cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(bad);
        return RAV_ERR_CUDA;
      }
      if (!hb) b.gtc = buf;
    }
    cudaFree(bad);
    bt->use_tc = true;
  }
  if (bt->graph) {  // the captured cycle holds the previous apply kernels
    cudaGraphExecDestroy(bt->graph);
    bt->graph = nullptr;
  }
  bt->cur_x.clear();  // descriptors are re-uploaded at the next bind
  RAV_TRY(build_phases(bt));
  RAV_CUDA(cudaGetLastError());
  return RAV_OK;
}

extern "C" int batch_set_coarse_residual_f32(rav_batch* bt, int enable, rav_stream stream) {
  if (!bt || (enable != 0 && enable != 1)) return RAV_ERR_ARG;
  if ((enable != 0) == bt->coarse_f32) return RAV_OK;
  cudaStream_t s = S(stream);
  RAV_CUDA(cudaStreamSynchronize(s));
  for (void* q : bt->c32_bufs) cudaFree(q);
  bt->c32_bufs.clear();
  for (BLevel& b : bt->lv) {
    b.sval32 = nullptr;
    b.x32 = nullptr;
  }
  bt->coarse_f32 = false;
  if (enable) {
    for (int p = 0; p < bt->nprob; ++p) {
      const int Lp = bt->mgs[p]->nlev;
      for (int d = 1; d <= Lp - 2; ++d) {  // depths below the finest that run residuals
        BLevel& b = bt->lv[bt->lv_first[p] + d];
        int64_t nval = 0;  // stored slots of the level's sliced-ELL copy
        RAV_CUDA(cudaMemcpy(&nval, b.sptr + b.nslice, sizeof(int64_t), cudaMemcpyDeviceToHost));
        float *v32 = nullptr, *x32 = nullptr;
        if (cudaMalloc(&v32, sizeof(float) * std::max<int64_t>(nval, 1)) != cudaSuccess) return RAV_ERR_CUDA;
        bt->c32_bufs.push_back(v32);
        if (cudaMalloc(&x32, sizeof(float) * b.g.n * bt->nrhs) != cudaSuccess) return RAV_ERR_CUDA;
        bt->c32_bufs.push_back(x32);
        if (nval) kb_vals_to_f32<<<(unsigned)((nval + 255) / 256), 256, 0, s>>>(b.sval, nval, v32);
        b.sval32 = v32;
        b.x32 = x32;
      }
    }
    RAV_CUDA(cudaGetLastError());
    bt->coarse_f32 = true;
  }
  if (bt->graph) {  // the captured cycle holds the previous residual kernels
    cudaGraphExecDestroy(bt->graph);
    bt->graph = nullptr;
  }
  bt->cur_x.clear();  // descriptors are re-uploaded at the next bind
  RAV_TRY(build_phases(bt));
  RAV_CUDA(cudaStreamSynchronize(s));
  return RAV_OK;
}

extern "C" int batch_set_transfers_f32(rav_batch* bt, int enable, rav_stream stream) {
  if (!bt || (enable != 0 && enable != 1)) return RAV_ERR_ARG;
  if (enable && (bt->prec != RAV_F32 || bt->elem != RAV_ELEM_Q2Q1)) return RAV_ERR_ARG;
  if ((enable != 0) == bt->xfer_f32) return RAV_OK;
  cudaStream_t s = S(stream);
  RAV_CUDA(cudaStreamSynchronize(s));
  for (void* q : bt->x32_bufs) cudaFree(q);
  bt->x32_bufs.clear();
  for (BLevel& b : bt->lv) {
    b.tab32 = XferTabT<float>{};
    b.xc32 = nullptr;
  }
  bt->xfer_f32 = false;
  if (enable) {
    for (int p = 0; p < bt->nprob; ++p) {
      const int Lp = bt->mgs[p]->nlev;
      for (int d = 0; d + 1 < Lp; ++d) {  // levels with a coarser one
        BLevel& b = bt->lv[bt->lv_first[p] + d];
        const int64_t mf = 2 * (int64_t)b.g.N + 1, mc = 2 * (int64_t)b.gc.N + 1;
        const int64_t n2 = 3 * mf, n1 = 2 * ((int64_t)b.g.N + 1), r2 = 7 * mc, r1 = 3 * ((int64_t)b.gc.N + 1);
        for (int a = 0; a < bt->dim; ++a) {
          float* w = nullptr;
          if (cudaMalloc(&w, sizeof(float) * (n2 + n1 + r2 + r1)) != cudaSuccess) return RAV_ERR_CUDA;
          bt->x32_bufs.push_back(w);
          kb_vals_to_f32<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(b.tab.pw2[a], n2, w);
          kb_vals_to_f32<<<(unsigned)((n1 + 255) / 256), 256, 0, s>>>(b.tab.pw1[a], n1, w + n2);
          kb_vals_to_f32<<<(unsigned)((r2 + 255) / 256), 256, 0, s>>>(b.tab.rw2[a], r2, w + n2 + n1);
          kb_vals_to_f32<<<(unsigned)((r1 + 255) / 256), 256, 0, s>>>(b.tab.rw1[a], r1, w + n2 + n1 + r2);
          XferTabT<float>& T = b.tab32;
          T.pc2[a] = b.tab.pc2[a];
          T.pk2[a] = b.tab.pk2[a];
          T.pc1[a] = b.tab.pc1[a];
          T.pk1[a] = b.tab.pk1[a];
          T.rc2[a] = b.tab.rc2[a];
          T.rk2[a] = b.tab.rk2[a];
          T.rc1[a] = b.tab.rc1[a];
          T.rk1[a] = b.tab.rk1[a];
          T.pw2[a] = w;
          T.pw1[a] = w + n2;
          T.rw2[a] = w + n2 + n1;
          T.rw1[a] = w + n2 + n1 + r2;
        }
        float* xc32 = nullptr;
        if (cudaMalloc(&xc32, sizeof(float) * b.gc.n * bt->nrhs) != cudaSuccess) return RAV_ERR_CUDA;
        bt->x32_bufs.push_back(xc32);
        b.xc32 = xc32;
      }
    }
    RAV_CUDA(cudaGetLastError());
    bt->xfer_f32 = true;
  }
  if (bt->graph) {  // the captured cycle holds the previous transfer kernels
    cudaGraphExecDestroy(bt->graph);
    bt->graph = nullptr;
  }
  bt->cur_x.clear();  // descriptors are re-uploaded at the next bind
  RAV_TRY(build_phases(bt));
  RAV_CUDA(cudaStreamSynchronize(s));
  return RAV_OK;
}

extern "C" int batch_transfers_f32(const rav_batch* bt) {
  if (!bt) return RAV_ERR_ARG;
  return bt->xfer_f32 ? 1 : 0;
}

extern "C" int batch_coarse_residual_f32(const rav_batch* bt) {
  if (!bt) return RAV_ERR_ARG;
  return bt->coarse_f32 ? 1 : 0;
}

extern "C" int batch_tensor_apply_levels(const rav_batch* bt) {
  if (!bt) return RAV_ERR_ARG;
  int n = 0;
  if (bt->use_tc)
    for (const BLevel& b : bt->lv) n += b.gtc != nullptr;
  return n;
}
